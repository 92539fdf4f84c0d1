"""Staircased tip geometry on a 3D Cartesian grid (test infrastructure only).

The paper solves on a 2D axisymmetric FEM mesh (Sec. 2.1, Fig. domains); the step here
uses the 3D Cartesian reading of the same geometry: cathode plane Gamma_cath at z=0
(phi=0, eq:bcf3), anode Gamma_ano at z = nz*dx (phi=V0, eq:bcf1), zero normal field on the
lateral vacuum boundary Gamma_vac (eq:bcf2), and a Cu tip made of solid cells held at phi=0.

Conventions (cell units; node (i,j,k) sits at (i,j,k)*dx, cell (i,j,k) spans [i,i+1)x...):
  * a cell is solid iff its centre c satisfies  rho_perp(c) <= r and c_z <= h - r,  or
    |c - (ax, ay, h - r)| <= r, with the axis at (ax, ay) = (nx/2, ny/2) and h the tip
    height including the hemispherical cap;
  * linear cell index  (k*ny + j)*nx + i;  linear node index (k*(ny+1) + j)*(nx+1) + i;
  * exposed faces are enumerated over vacuum cells in linear order and, per cell, over the
    directions -x,+x,-y,+y,-z,+z (codes 0..5); a face exists where the neighbour in that
    direction is solid, or for direction -z at k=0 (the cathode plane under a vacuum cell).
"""
import numpy as np

DIRS = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, 0], [0, 1, 0], [0, 0, -1], [0, 0, 1]], dtype=np.int64)


class Grid:
    def __init__(self, nx, ny, nz, dx, tip_radius, tip_height):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.dx = float(dx)
        self.r_c = float(tip_radius) / float(dx)
        self.h_c = float(tip_height) / float(dx)
        self.ax = self.nx / 2.0
        self.ay = self.ny / 2.0
        self.ncell = self.nx * self.ny * self.nz
        self.nnode = (self.nx + 1) * (self.ny + 1) * (self.nz + 1)
        self.solid = self._solid_mask()
        self._faces()

    # -- cells ---------------------------------------------------------------------------
    def _solid_mask(self):
        k, j, i = np.meshgrid(np.arange(self.nz), np.arange(self.ny), np.arange(self.nx), indexing="ij")
        cx, cy, cz = i + 0.5, j + 0.5, k + 0.5
        rho2 = (cx - self.ax) ** 2 + (cy - self.ay) ** 2
        zc = self.h_c - self.r_c
        shaft = (rho2 <= self.r_c ** 2) & (cz <= zc)
        cap = rho2 + (cz - zc) ** 2 <= self.r_c ** 2
        return shaft | cap

    def cell_index(self, i, j, k):
        return (np.asarray(k) * self.ny + np.asarray(j)) * self.nx + np.asarray(i)

    def node_index(self, i, j, k):
        return (np.asarray(k) * (self.ny + 1) + np.asarray(j)) * (self.nx + 1) + np.asarray(i)

    # -- faces ---------------------------------------------------------------------------
    def _faces(self):
        """Vacuum cells in linear order, per cell the directions 0..5 in order (array form of the
        double loop: a face exists toward a solid neighbour, or toward z < 0 from a k = 0 cell)."""
        nx, ny, nz = self.nx, self.ny, self.nz
        solid = self.solid
        vac = ~solid
        has = np.zeros((nz, ny, nx, 6), dtype=bool)
        own = np.full((nz, ny, nx, 6), -1, dtype=np.int64)
        cidx = np.arange(self.ncell, dtype=np.int64).reshape(nz, ny, nx)
        for d in range(6):
            di, dj, dk = DIRS[d]
            nb_solid = np.zeros_like(solid)
            nb_idx = np.full(solid.shape, -1, dtype=np.int64)
            src = (slice(max(dk, 0), nz + min(dk, 0)), slice(max(dj, 0), ny + min(dj, 0)), slice(max(di, 0), nx + min(di, 0)))
            dst = (slice(max(-dk, 0), nz + min(-dk, 0)), slice(max(-dj, 0), ny + min(-dj, 0)), slice(max(-di, 0), nx + min(-di, 0)))
            nb_solid[dst] = solid[src]
            nb_idx[dst] = cidx[src]
            has[..., d] = vac & nb_solid
            own[..., d] = np.where(nb_solid, nb_idx, -1)
            if d == 4:
                has[0, :, :, 4] = vac[0]            # cathode plane under a vacuum cell
                own[0, :, :, 4] = -1
        flat = has.reshape(-1, 6)
        cells, dirs = np.nonzero(flat)
        self.face_vcell = cells.astype(np.int64)
        self.face_dir = dirs.astype(np.int64)
        self.face_owner = own.reshape(-1, 6)[cells, dirs]
        self.nface = len(cells)
        self.face_key = self.face_vcell * 6 + self.face_dir     # ascending by construction

    def face_cell_ijk(self, f):
        c = self.face_vcell[f]
        return c % self.nx, (c // self.nx) % self.ny, c // (self.nx * self.ny)

    def face_geometry(self, f):
        """(axis, sign, plane) of face f: the face lies in the plane x_axis = plane and its
        normal (from solid to vacuum) is sign * e_axis; returns also the vacuum cell ijk."""
        i, j, k = self.face_cell_ijk(f)
        d = self.face_dir[f]
        axis = d // 2
        ijk = np.array([i, j, k])
        if d % 2 == 0:          # solid on the - side: plane at the cell's lower boundary
            plane = ijk[axis]
            sign = 1
        else:                    # solid on the + side: plane at the cell's upper boundary
            plane = ijk[axis] + 1
            sign = -1
        return int(axis), int(sign), int(plane), ijk

    def face_lookup(self, vcell, d):
        """Face id of (vacuum cell, direction) by binary search in the face key list; -1 if absent."""
        key = np.asarray(vcell, dtype=np.int64) * 6 + np.asarray(d, dtype=np.int64)
        pos = np.searchsorted(self.face_key, key)
        pos = np.minimum(pos, self.nface - 1)
        return np.where(self.face_key[pos] == key, pos, -1)

    # -- nodes ---------------------------------------------------------------------------
    def dirichlet_mask(self):
        """Nodes fixed by eq:bcf1/eq:bcf3: z=0 plane, z=nz plane, every corner of a solid cell."""
        nx, ny, nz = self.nx, self.ny, self.nz
        m = np.zeros((nz + 1, ny + 1, nx + 1), dtype=bool)
        m[0] = True
        m[nz] = True
        s = self.solid
        for dk in (0, 1):
            for dj in (0, 1):
                for di in (0, 1):
                    m[dk:dk + nz, dj:dj + ny, di:di + nx] |= s
        return m

    def dirichlet_values(self, V0):
        v = np.zeros((self.nz + 1, self.ny + 1, self.nx + 1))
        v[self.nz] = V0
        return v

    def apex_faces(self):
        """+z tip faces of the highest owner cells touching the axis: the apex (calibration)."""
        nx, ny = self.nx, self.ny
        ai, aj = int(np.floor(self.ax)), int(np.floor(self.ay))
        cand = []
        for f in range(self.nface):
            if self.face_dir[f] != 4 or self.face_owner[f] < 0:
                continue
            o = self.face_owner[f]
            oi, oj, ok = o % nx, (o // nx) % ny, o // (nx * ny)
            if oi in (ai - 1, ai) and oj in (aj - 1, aj):
                cand.append((ok, f))
        top = max(c[0] for c in cand)
        return np.array([f for ok, f in cand if ok == top], dtype=np.int64)
