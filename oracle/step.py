"""One coupled PIC-MCC step (test infrastructure only).

Order (Sec. 2.3.1 and Fig. newpic; the paper prints no pseudocode, this is the reading):
  a1 emission from every exposed face (field from phi^n, temperature of the owner cell)
  a2 surface injection: evaporation, then sputtering from the previous step's ion impacts
  a3 gather + leapfrog push of every SP (new ones included) + boundary removal / ion impacts
     (Cu+ and Cu2+ alike; with an external circuit, prm circuit_R and circuit_C > 0: then the
     Shockley-Ramo current of the pushed e-, Cu+ and Cu2+ and one Euler step of the RC circuit;
     the step's Poisson solve holds the anode at the new V_gap)
  a4 stable cell sort of every species (survivors in previous order); with prm merge_max > 0,
     SP merging in the over-full cells
  a5 impact ionization MCC (with prm "ion2": the Cu2+ channels of Table colls, double
     ionization of Cu inside the same pass and then Cu+ + e -> Cu2+ + 2e; with prm "elastic":
     then e-Cu and Cu-Cu elastic collisions and Cu+-Cu charge exchange; with prm "coulomb": then
     e-e, e-Cu+ and Cu+-Cu+ Coulomb collisions, and with "ion2" also e-Cu2+, Cu+-Cu2+ and
     Cu2+-Cu2+; all on the sorted SPs), a6 direct field ionization
  a7 fixed-point charge deposit, a8 Poisson solve, a9 node field
  a10 every n_heat steps: continuity + heat on the tip cells

New SPs take consecutive ids in this order: emitted electrons (face order), evaporated
neutrals (face order), sputtered neutrals (face order), MCC products (pair order: ion,
scattered electron, secondary electron; then the double ionizations in pair order: Cu2+,
scattered electron, two secondary electrons; then the Cu+ ionizations: Cu2+, scattered
electron, secondary electron), elastic products, DFI products (neutral order: ion, electron).
Within each species, new SPs are appended after the existing ones in the same order.
"""
import math

import numpy as np

from . import circuit, collide, coulomb, elastic, emission, field, heat, merge, particles as P, philox, surface
from . import constants as C

E_, N_, I_, J_ = "e", "n", "i", "j"
SPECIES = {E_: (-1, C.M_E), N_: (0, C.M_CU), I_: (1, C.M_CU), J_: (2, C.M_CU)}
IONS = (I_, J_)
F32 = np.float32


class State:
    def __init__(self, grid, prm, species, phi, T=None):
        self.grid = grid
        self.prm = dict(prm)
        self.sp = {k: {f: np.asarray(v[f]).astype(P.DTYPES[f]).copy() for f in P.FIELDS} for k, v in species.items()}
        for k in SPECIES:               # Cu2+ (and any species not given) starts empty
            self.sp.setdefault(k, P.empty())
        self.phi = np.asarray(phi, dtype=np.float64).copy()
        self.E = field.efield(grid, self.phi)
        ncv = int(grid.solid.sum())
        self.T = np.full(ncv, prm["T0"]) if T is None else np.asarray(T, dtype=np.float64).copy()
        nf = grid.nface
        self.acc_evap = np.zeros(nf)
        self.acc_sput = np.zeros(nf, dtype=np.int64)
        self.acc_Eb = np.zeros(nf, dtype=np.int64)
        self.acc_Es = np.zeros(nf, dtype=np.int64)
        self.acc_heat = np.zeros(nf)          # P_N + P_vap energy [J] over the heat interval
        self.acc_charge = np.zeros(nf)        # emitted charge [C] over the heat interval
        self.step = int(prm.get("step0", 0))
        self.next_id = int(prm.get("next_id", 0))
        self.count = {}
        self.off = {}
        for k in self.sp:
            self.sp[k], self.off[k] = P.stable_sort(grid, self.sp[k])
        self.Q = None
        self.circuit = prm.get("circuit_R", 0) > 0 and prm.get("circuit_C", 0) > 0
        self.V_gap, self.I_gap, self.I_tot = float(prm["V0"]), 0.0, 0.0
        self.E0 = None


def face_temperature(st):
    g = st.grid
    cells = np.nonzero(g.solid.ravel())[0]
    index = -np.ones(g.ncell, dtype=np.int64)
    index[cells] = np.arange(len(cells))
    T = np.full(g.nface, st.prm["T0"])
    tip = g.face_owner >= 0
    T[tip] = st.T[index[g.face_owner[tip]]]
    return T


def face_radius_nm(g, prm):
    return np.where(g.face_owner >= 0, prm["tip_radius"] * 1e9, np.inf)


def face_point(g, f, ua, ub):
    """Position (f32, cell units) of a point on face f with tangential fractions ua, ub."""
    axis, sign, plane, ijk = g.face_geometry(f)
    t = [a for a in range(3) if a != axis]
    pos = [F32(0), F32(0), F32(0)]
    pn = F32(plane)
    pos[axis] = pn if sign > 0 else np.nextafter(pn, F32(-np.inf))
    for a, u in zip(t, (ua, ub)):
        v = F32(ijk[a]) + F32(u)
        pos[a] = min(v, np.nextafter(F32(ijk[a] + 1), F32(-np.inf)))
    return pos, axis, sign, t


def emit(st, J):
    """a1: N_f = floor(lam) + [U < lam - floor(lam)], lam = J A dt / (e w_min); new electrons at rest."""
    g, prm, n = st.grid, st.prm, st.step
    A = g.dx * g.dx
    lam = J * A * prm["dt"] / (C.E_CHARGE * prm["w_min"])
    base = np.floor(lam)
    U = philox.uniform(prm["seed"], philox.EMIT, np.arange(g.nface), n, 0)
    N = base.astype(np.int64) + (U < lam - base)
    new = []
    for f in np.nonzero(N)[0]:
        for j in range(int(N[f])):
            ua = philox.uniform(prm["seed"], philox.EMIT, f, n, 1 + 2 * j)
            ub = philox.uniform(prm["seed"], philox.EMIT, f, n, 2 + 2 * j)
            pos, _, _, _ = face_point(g, f, ua, ub)
            new.append({"x": pos[0], "y": pos[1], "z": pos[2], "vx": F32(0), "vy": F32(0), "vz": F32(0),
                        "w": np.int32(1), "id": np.uint64(st.next_id)})
            st.next_id += 1
    return N, collide._append(new)


def cell_sp_counts(st):
    return sum(np.diff(st.off[k]) for k in st.off)


def inject(st):
    """a2: evaporation and sputter injection of neutrals (Sec. 2.3.1-2.3.3)."""
    g, prm, n = st.grid, st.prm, st.step
    A = g.dx * g.dx
    Tf = face_temperature(st)
    flux = surface.evaporation_flux(Tf)
    st.acc_evap += flux * A * prm["dt"]
    st.acc_heat -= C.E_VAP_EV * C.E_CHARGE * flux * A * prm["dt"]
    ncnt = cell_sp_counts(st)
    Vc = g.dx ** 3
    wmin = prm["w_min"]
    new_evap, new_sput = [], []
    for f in range(g.nface):
        ncell = ncnt[g.face_vcell[f]] / Vc
        # evaporation
        Ninj = math.floor(st.acc_evap[f])
        if Ninj >= 1:
            wu = surface.injection_weight_units(ncell, Ninj, wmin, prm["w_max_units"])
            nsp = int(math.floor(st.acc_evap[f] / (wu * wmin)))
            st.acc_evap[f] -= nsp * wu * wmin
            m = C.M_CU
            sig = math.sqrt(C.K_B * Tf[f] / m)
            for j in range(nsp):
                u = philox.uniform(prm["seed"], philox.EVAP, f, n, 8 * j + np.arange(5))
                pos, axis, sign, t = face_point(g, f, u[0], u[1])
                vn = math.sqrt(-2.0 * C.K_B * Tf[f] / m * math.log(u[2]))
                r = sig * math.sqrt(-2.0 * math.log(u[3]))
                vel = [0.0, 0.0, 0.0]
                vel[axis] = sign * vn
                vel[t[0]] = r * math.cos(2.0 * math.pi * u[4])
                vel[t[1]] = r * math.sin(2.0 * math.pi * u[4])
                new_evap.append({"x": pos[0], "y": pos[1], "z": pos[2], "vx": F32(vel[0]), "vy": F32(vel[1]),
                                 "vz": F32(vel[2]), "w": np.int32(wu), "id": np.uint64(st.next_id)})
                st.next_id += 1
    for f in range(g.nface):
        ncell = ncnt[g.face_vcell[f]] / Vc
        lam = st.acc_sput[f] * 2.0 ** -surface.SPUT_FRAC_BITS
        Ninj = math.floor(lam)
        if Ninj >= 1:
            wu = surface.injection_weight_units(ncell, Ninj, wmin, prm["w_max_units"])
            nsp = int(math.floor(lam / (wu * wmin)))
            # the accumulator counts real atoms in 2^-24 units: remove the nsp*wu*w_min atoms
            # the new SPs carry (Sec. 2.3.3), rounded down to the accumulator's resolution
            st.acc_sput[f] -= int(math.floor(nsp * wu * wmin * 2.0 ** surface.SPUT_FRAC_BITS))
            for j in range(nsp):
                u = philox.uniform(prm["seed"], philox.SPUT, f, n, 8 * j + np.arange(5))
                pos, axis, sign, t = face_point(g, f, u[0], u[1])
                Es = surface.thompson_energy(u[2])
                v = math.sqrt(2.0 * Es * C.E_CHARGE / C.M_CU)
                ct = u[3]
                st_ = math.sqrt(max(0.0, 1.0 - ct * ct))
                ph = 2.0 * math.pi * u[4]
                vel = [0.0, 0.0, 0.0]
                vel[axis] = sign * v * ct
                vel[t[0]] = v * st_ * math.cos(ph)
                vel[t[1]] = v * st_ * math.sin(ph)
                new_sput.append({"x": pos[0], "y": pos[1], "z": pos[2], "vx": F32(vel[0]), "vy": F32(vel[1]),
                                 "vz": F32(vel[2]), "w": np.int32(wu), "id": np.uint64(st.next_id)})
                st.next_id += 1
                st.acc_Es[f] += int(math.floor(wu * wmin * Es * 2.0 ** surface.ENERGY_FRAC_BITS))
    return collide._append(new_evap), collide._append(new_sput)


def record_impacts(st, impacts):
    wmin = st.prm["w_min"]
    for (f, E, w) in impacts:
        st.acc_sput[f] += int(math.floor(w * wmin * surface.sputter_yield(E) * 2.0 ** surface.SPUT_FRAC_BITS))
        st.acc_Eb[f] += int(math.floor(w * wmin * E * 2.0 ** surface.ENERGY_FRAC_BITS))


def push_all(st):
    """a3 for every species; returns {species: alive mask} after applying the new state."""
    g, prm = st.grid, st.prm
    dtdx = F32(prm["dt"] / g.dx)
    alive = {}
    for k, (Z, m) in SPECIES.items():
        sp_ = st.sp[k]
        qmdt = P.kick_factor(Z, m, prm["dt"]) if Z != 0 else 0.0
        new = P.push_f32(sp_, st.E, qmdt, dtdx)
        a, impacts = P.boundary(g, sp_, new, k in IONS, m)
        if k in IONS:
            record_impacts(st, impacts)
        for c, v in zip(("x", "y", "z", "vx", "vy", "vz"), new):
            sp_[c] = v.astype(np.float32)
        alive[k] = a
        st.count["removed_" + k] = int((~a).sum())
        if k == I_:
            st.count["ion_impacts"] = len(impacts)
        elif k == J_:
            st.count["ion_impacts"] += len(impacts)
    return alive


def circuit_update(st, alive):
    """The circuit passage of Sec. 2.3.1: I_gap of the pushed e-, Cu+ and Cu2+ still in the domain,
    then V_gap <- V_gap + dt/C (I_tot - I_gap) with I_tot = (V0 - V_gap)/R."""
    prm = st.prm
    if st.E0 is None:
        st.E0 = circuit.unit_field(st.grid)
    charged = [(SPECIES[k][0], P.take(st.sp[k], np.nonzero(alive[k])[0])) for k in (E_, I_, J_)]
    st.I_gap = circuit.gap_current(st.E0, charged, prm["w_min"])
    st.V_gap, st.I_tot = circuit.circuit_step(st.V_gap, st.I_gap, prm["V0"], prm["circuit_R"], prm["circuit_C"],
                                              prm["dt"])


def deposit_all(st):
    g = st.grid
    Q = P.deposit(g, st.sp[E_], -1)
    Q = P.deposit(g, st.sp[I_], 1, Q=Q)
    Q = P.deposit(g, st.sp[J_], 2, Q=Q)
    return Q


def solve_field(st):
    g, prm = st.grid, st.prm
    st.Q = deposit_all(st)
    f = field.rhs_from_charge(g, st.Q, prm["w_min"])
    st.phi = field.solve_poisson(g, st.V_gap if st.circuit else prm["V0"], f)
    st.E = field.efield(g, st.phi)


def step(st, emission_fn=None):
    g, prm = st.grid, st.prm
    A = g.dx * g.dx
    # a1
    Fv = field.face_field(g, st.phi)
    Tf = face_temperature(st)
    Rf = face_radius_nm(g, prm)
    if emission_fn is None:
        J, PN = emission.current_density_fixed(Fv * 1e-9, Tf, prm["work_function"], Rf)
    else:
        J, PN = emission_fn(Fv * 1e-9, Tf, prm["work_function"], Rf)
    st.last_J, st.last_F = J, Fv
    Nemit, new_e = emit(st, J)
    st.acc_heat += PN * A * prm["dt"]
    st.acc_charge += J * A * prm["dt"]
    st.count["emitted"] = int(Nemit.sum())
    # a2
    new_ev, new_sp = inject(st)
    st.count["evaporated"] = P.count(new_ev)
    st.count["sputtered"] = P.count(new_sp)
    st.sp[E_] = P.concat(st.sp[E_], new_e)
    st.sp[N_] = P.concat(P.concat(st.sp[N_], new_ev), new_sp)
    # a3
    alive = push_all(st)
    if st.circuit:
        circuit_update(st, alive)
    # a4
    for k in st.sp:
        st.sp[k], st.off[k] = P.stable_sort(g, st.sp[k], alive[k])
    if prm.get("merge_max", 0) > 0:
        st.count["merged"] = sum(merge.merge_species(st.sp[k], st.off[k], prm["merge_max"], prm["w_max_units"])
                                 for k in (E_, N_, I_, J_))
    # a5
    ids = collide.Counter(st.next_id)
    ion2 = bool(prm.get("ion2"))
    mcc = collide.impact_ionization(g, prm, st.sp[E_], st.off[E_], st.sp[N_], st.off[N_], st.step, ids, double=ion2)
    ni, ne, st.count["impact_ionizations"] = mcc[:3]
    nj, ne_d, nj_iz, ne_iz = P.empty(), P.empty(), P.empty(), P.empty()
    if ion2:
        nj, ne_d, st.count["double_ionizations"] = mcc[3:]
        nj_iz, ne_iz, st.count["ion_ionizations"] = collide.ion_ionization(g, prm, st.sp[E_], st.off[E_], st.sp[I_],
                                                                           st.off[I_], st.step, ids)
    el_e, el_i = P.empty(), P.empty()
    if prm.get("elastic"):
        el_e, el_n1, st.count["elastic_en"] = elastic.elastic_en(g, prm, st.sp[E_], st.off[E_], st.sp[N_], st.off[N_],
                                                                 st.step, ids)
        el_n2, st.count["elastic_nn"] = elastic.elastic_nn(g, prm, st.sp[N_], st.off[N_], st.step, ids)
        el_i, el_n3, st.count["charge_exchanges"] = elastic.charge_exchange(g, prm, st.sp[I_], st.off[I_], st.sp[N_],
                                                                            st.off[N_], st.step, ids)
        st.sp[N_] = P.concat(P.concat(P.concat(st.sp[N_], el_n1), el_n2), el_n3)
    if prm.get("coulomb"):
        st.count["coulomb_ee"] = coulomb.coulomb_ee(g, prm, st.sp[E_], st.off[E_], st.step)
        st.count["coulomb_ei"] = coulomb.coulomb_ei(g, prm, st.sp[E_], st.off[E_], st.sp[I_], st.off[I_], st.step)
        st.count["coulomb_ii"] = coulomb.coulomb_ii(g, prm, st.sp[I_], st.off[I_], st.step)
        if ion2:
            st.count["coulomb_ej"] = coulomb.coulomb_ej(g, prm, st.sp[E_], st.off[E_], st.sp[J_], st.off[J_], st.step)
            st.count["coulomb_ij"] = coulomb.coulomb_ij(g, prm, st.sp[I_], st.off[I_], st.sp[J_], st.off[J_], st.step)
            st.count["coulomb_jj"] = coulomb.coulomb_jj(g, prm, st.sp[J_], st.off[J_], st.step)
    # a6
    ni2, ne2, ev2 = collide.field_ionization(g, prm, st.sp[N_], st.E, st.step, ids)
    st.count["field_ionizations"] = ev2
    st.next_id = ids.next_id
    st.sp[I_] = P.concat(P.concat(P.concat(st.sp[I_], ni), el_i), ni2)
    st.sp[E_] = P.concat(P.concat(P.concat(P.concat(P.concat(st.sp[E_], ne), ne_d), ne_iz), el_e), ne2)
    st.sp[J_] = P.concat(P.concat(st.sp[J_], nj), nj_iz)
    # a7-a9
    solve_field(st)
    # a10
    st.step += 1
    nh = prm.get("n_heat", 0)
    if nh and st.step % nh == 0:
        heat_update(st)


def heat_update(st):
    g, prm = st.grid, st.prm
    dth = prm["dt"] * prm["n_heat"]
    Eb = (st.acc_Eb - st.acc_Es).astype(np.float64) * 2.0 ** -surface.ENERGY_FRAC_BITS * C.E_CHARGE
    Pheat = (st.acc_heat + Eb) / dth
    Icur = st.acc_charge / dth
    st.T, st.joule = heat.heat_step(g, st.T, Pheat, Icur, dth, prm["T0"])
    st.acc_heat[:] = 0
    st.acc_charge[:] = 0
    st.acc_Eb[:] = 0
    st.acc_Es[:] = 0
