"""Particle kernels of the PIC step (test infrastructure only), Sec. 2.2.

Superparticles (SPs) of one species are a dict of arrays:
    x, y, z   float32, position in cell units (x/dx), inside [0,nx) x [0,ny) x [0,nz)
    vx,vy,vz  float32, velocity in m/s (for the leapfrog: v^{n-1/2})
    w         int32, weight in units of w_min (Sec. 2.3.2: weights are multiples of w_min)
    id        uint64, creation id; keys every random draw of the SP

Precision: the paper fixes none.  The push is evaluated in float32 with a fixed operation
order (the kernel's precision) because the new cell keys, boundary events and deposits are
integer decisions taken from the pushed f32 positions; positions in float64 are also
provided (`push_f64`) for the float tolerance check.  Boundary crossings are resolved in
float64 (Amanatides-Woo traversal) from the two f32 end points.
"""
import numpy as np

from . import constants as C

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "w", "id")
DTYPES = {"x": np.float32, "y": np.float32, "z": np.float32, "vx": np.float32, "vy": np.float32,
          "vz": np.float32, "w": np.int32, "id": np.uint64}

F32 = np.float32


def empty():
    return {k: np.zeros(0, dtype=DTYPES[k]) for k in FIELDS}


def take(sp_, idx):
    return {k: sp_[k][idx] for k in FIELDS}


def concat(a, b):
    return {k: np.concatenate([a[k], b[k]]).astype(DTYPES[k]) for k in FIELDS}


def count(sp_):
    return len(sp_["x"])


# --------------------------------------------------------------------------------------
# gather (cloud-in-cell) -- Sec. 2.2 leaves the interpolation to the FEMOCS paper; CIC is
# the reading used here: trilinear weights from the fractional cell position.
# --------------------------------------------------------------------------------------
def _lerp(a, b, t):
    return a + t * (b - a)          # float32: one rounding per operation, no fused multiply-add


def gather(E, x, y, z):
    """E at positions (f32, cell units) by nested lerps: x, then y, then z."""
    i = np.floor(x).astype(np.int64)
    j = np.floor(y).astype(np.int64)
    k = np.floor(z).astype(np.int64)
    fx = (x - i.astype(F32)).astype(F32)[:, None]
    fy = (y - j.astype(F32)).astype(F32)[:, None]
    fz = (z - k.astype(F32)).astype(F32)[:, None]
    c00 = _lerp(E[k, j, i], E[k, j, i + 1], fx)
    c10 = _lerp(E[k, j + 1, i], E[k, j + 1, i + 1], fx)
    c01 = _lerp(E[k + 1, j, i], E[k + 1, j, i + 1], fx)
    c11 = _lerp(E[k + 1, j + 1, i], E[k + 1, j + 1, i + 1], fx)
    c0 = _lerp(c00, c10, fy)
    c1 = _lerp(c01, c11, fy)
    return _lerp(c0, c1, fz)


def kick_factor(charge_e, mass, dt):
    """f32(q/m * dt), evaluated in float64 and rounded once."""
    return F32(charge_e * C.E_CHARGE / mass * dt)


def push_f32(sp_, E, qmdt, dtdx):
    """Leapfrog (Sec. 2.2): v^{n+1/2} = v^{n-1/2} + (q/m) E(x^n) dt; x^{n+1} = x^n + v^{n+1/2} dt.
    Neutral species (qmdt == 0) move ballistically.  Returns new (x, y, z, vx, vy, vz) f32."""
    x, y, z = sp_["x"], sp_["y"], sp_["z"]
    vx, vy, vz = sp_["vx"].copy(), sp_["vy"].copy(), sp_["vz"].copy()
    if qmdt != 0 and len(x):
        e = gather(E, x, y, z)
        vx = vx + F32(qmdt) * e[:, 0]
        vy = vy + F32(qmdt) * e[:, 1]
        vz = vz + F32(qmdt) * e[:, 2]
    dtdx = F32(dtdx)
    return x + vx * dtdx, y + vy * dtdx, z + vz * dtdx, vx, vy, vz


def push_f64(sp_, E64, qm_dt64, dtdx64):
    """The same leapfrog in float64 with a float64 node field (tolerance reference)."""
    x, y, z = (sp_[c].astype(np.float64) for c in ("x", "y", "z"))
    vx, vy, vz = (sp_[c].astype(np.float64) for c in ("vx", "vy", "vz"))
    if qm_dt64 != 0 and len(x):
        i, j, k = np.floor(x).astype(int), np.floor(y).astype(int), np.floor(z).astype(int)
        fx, fy, fz = x - i, y - j, z - k
        e = np.zeros((len(x), 3))
        for dk in (0, 1):
            for dj in (0, 1):
                for di in (0, 1):
                    wgt = (fx if di else 1 - fx) * (fy if dj else 1 - fy) * (fz if dk else 1 - fz)
                    e += wgt[:, None] * E64[k + dk, j + dj, i + di]
        vx = vx + qm_dt64 * e[:, 0]
        vy = vy + qm_dt64 * e[:, 1]
        vz = vz + qm_dt64 * e[:, 2]
    return x + vx * dtdx64, y + vy * dtdx64, z + vz * dtdx64, vx, vy, vz


# --------------------------------------------------------------------------------------
# boundaries -- Sec. 2.2: SPs that cross Gamma_cath, Gamma_vac or Gamma_ano are removed.
# --------------------------------------------------------------------------------------
EV_NONE, EV_SOLID, EV_CATHODE, EV_ANODE, EV_LATERAL = 0, 1, 2, 3, 4


def first_event(grid, p0, p1):
    """First boundary event on the straight segment p0 -> p1 (cell units, float64).

    Cells are traversed in the order their boundaries are crossed (ties: x before y before
    z); the first cell entered that is solid or outside the domain ends the traversal.
    Returns (event, vacuum cell left, direction code 0..5 of the crossing)."""
    n = (grid.nx, grid.ny, grid.nz)
    c = np.floor(p0).astype(np.int64)
    # end cell clamped to [-1, n]: leaving the domain is an event before any clamped cell
    ce = np.array([int(min(max(np.floor(p1[a]), -1.0), n[a])) for a in range(3)], dtype=np.int64)
    d = p1 - p0
    while not np.array_equal(c, ce):
        best_a, best_t = -1, 0.0
        for a in range(3):
            if c[a] == ce[a]:
                continue
            bnd = c[a] + 1 if ce[a] > c[a] else c[a]
            t = (float(bnd) - p0[a]) / d[a]
            if best_a < 0 or t < best_t:
                best_a, best_t = a, t
        a = best_a
        step = 1 if ce[a] > c[a] else -1
        prev = c.copy()
        c[a] += step
        dcode = 2 * a + (1 if step > 0 else 0)
        vcell = grid.cell_index(*prev)
        if c[a] < 0 or c[a] >= n[a]:
            if a == 2:
                return (EV_CATHODE if step < 0 else EV_ANODE), vcell, dcode
            return EV_LATERAL, vcell, dcode
        if grid.solid[c[2], c[1], c[0]]:
            return EV_SOLID, vcell, dcode
    return EV_NONE, -1, -1


def boundary(grid, sp_, new, is_ion, mass):
    """Apply the boundary test to pushed SPs.  Returns (alive mask, impacts) where impacts is a
    list of (face id, energy eV, weight) for ions that hit the tip or the cathode plane."""
    x0, y0, z0 = sp_["x"], sp_["y"], sp_["z"]
    x1, y1, z1, vx, vy, vz = new
    n = len(x0)
    alive = np.ones(n, dtype=bool)
    impacts = []
    c0 = np.stack([np.floor(x0), np.floor(y0), np.floor(z0)], 1).astype(np.int64)
    finite = np.isfinite(x1) & np.isfinite(y1) & np.isfinite(z1)
    alive &= finite
    lim = np.array([grid.nx, grid.ny, grid.nz], dtype=np.float64)
    c1 = np.clip(np.floor(np.stack([np.where(finite, x1, 0), np.where(finite, y1, 0), np.where(finite, z1, 0)], 1)
                          .astype(np.float64)), -1.0, lim).astype(np.int64)
    moved = np.nonzero(np.any(c0 != c1, axis=1) & finite)[0]
    for p in moved:
        ev, vcell, dcode = first_event(grid,
                                       np.array([x0[p], y0[p], z0[p]], dtype=np.float64),
                                       np.array([x1[p], y1[p], z1[p]], dtype=np.float64))
        if ev == EV_NONE:
            continue
        alive[p] = False
        if is_ion and ev in (EV_SOLID, EV_CATHODE):
            face = int(grid.face_lookup(vcell, dcode))
            v2 = float(vx[p]) ** 2 + float(vy[p]) ** 2 + float(vz[p]) ** 2
            energy = 0.5 * mass * v2 / C.E_CHARGE
            impacts.append((face, energy, int(sp_["w"][p])))
    return alive, impacts


# --------------------------------------------------------------------------------------
# cell sort -- Sec. 2.2: collisions pair SPs that share a cell, so SPs are grouped by cell.
# --------------------------------------------------------------------------------------
def cell_keys(grid, sp_):
    i = np.floor(sp_["x"]).astype(np.int64)
    j = np.floor(sp_["y"]).astype(np.int64)
    k = np.floor(sp_["z"]).astype(np.int64)
    return grid.cell_index(i, j, k)


def stable_sort(grid, sp_, alive=None):
    """Stable sort of the surviving SPs (alive and weight > 0) by cell; returns (sorted SPs,
    offsets[ncell+1])."""
    keys = cell_keys(grid, sp_)
    keep = sp_["w"] > 0 if alive is None else (alive & (sp_["w"] > 0))
    idx = np.nonzero(keep)[0]
    order = idx[np.argsort(keys[idx], kind="stable")]
    out = take(sp_, order)
    cnt = np.bincount(keys[order], minlength=grid.ncell)
    off = np.zeros(grid.ncell + 1, dtype=np.int64)
    off[1:] = np.cumsum(cnt)
    return out, off


# --------------------------------------------------------------------------------------
# charge deposit -- the density rho of eq:poi, cloud-in-cell with quantised fractions.
# --------------------------------------------------------------------------------------
def deposit(grid, sp_, charge_e, frac_bits=10, Q=None):
    """Q_node += Z w prod_axes(W_axis), W = 2^F - q on the lower node and q on the upper node,
    q = floor(frac(x) 2^F) from the f32 position.  Exact int64 (units e w_min 2^-3F)."""
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    if Q is None:
        Q = np.zeros((nz + 1, ny + 1, nx + 1), dtype=np.int64)
    if count(sp_) == 0 or charge_e == 0:
        return Q
    one = 1 << frac_bits
    q, base = [], []
    for c in ("x", "y", "z"):
        v = sp_[c]
        fl = np.floor(v)
        base.append(fl.astype(np.int64))
        q.append(np.floor((v - fl).astype(np.float64) * one).astype(np.int64))
    zw = np.int64(charge_e) * sp_["w"].astype(np.int64)
    flat = Q.reshape(-1)
    for dk in (0, 1):
        wz = q[2] if dk else one - q[2]
        for dj in (0, 1):
            wy = q[1] if dj else one - q[1]
            for di in (0, 1):
                wx = q[0] if di else one - q[0]
                node = grid.node_index(base[0] + di, base[1] + dj, base[2] + dk)
                np.add.at(flat, node, zw * wx * wy * wz)
    return Q
