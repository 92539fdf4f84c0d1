"""Electrostatics on the node grid (test infrastructure only).

Restates eq:poi, nabla^2 phi = -rho/eps0, with the boundary conditions eq:bcf1 (phi=V0 on the
anode plane z=nz), eq:bcf2 (zero normal field on the lateral vacuum boundary, read as the
boundary's own normal: the text's "cathode surface normal" is garbled) and eq:bcf3 (phi=0 on
the cathode plane and on every corner node of a solid tip cell).

Discretisation (the paper's FEM is replaced by finite differences on the configs' grid):
    (A phi)_n = (6 phi_n - sum of the 6 neighbours) / dx^2 = rho_n / eps0   for free nodes n,
where a neighbour across a lateral boundary is replaced by its mirror image (phi_{-1}=phi_1),
which is the finite-volume form on the half control volume at the boundary.  The node charge
density is rho_n = Q_n / V_n with V_n = dx^3 halved for each lateral boundary the node lies on.

The oracle solves the free-node system with plain conjugate gradients (scipy) to a relative
residual of 1e-13 on its symmetric finite-volume form (rows scaled by V_n/dx^3, Dirichlet
values moved to the right-hand side): no multigrid, no mixed precision.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import constants as C


def _mirror(idx, n):
    """Index of the mirror neighbour across a lateral boundary (n = number of cells)."""
    idx = np.where(idx < 0, -idx, idx)
    return np.where(idx > n, 2 * n - idx, idx)


def node_volume(grid):
    nx, ny, nz, dx = grid.nx, grid.ny, grid.nz, grid.dx
    fx = np.ones(nx + 1); fx[0] = fx[-1] = 0.5
    fy = np.ones(ny + 1); fy[0] = fy[-1] = 0.5
    return dx ** 3 * np.ones((nz + 1, 1, 1)) * fy[None, :, None] * fx[None, None, :]


def apply_operator(grid, phi):
    """(6 phi - sum neighbours)/dx^2 at every node, mirror across lateral boundaries;
    z neighbours outside [0, nz] are not needed (those planes are Dirichlet) and read 0."""
    nx, ny, nz, dx = grid.nx, grid.ny, grid.nz, grid.dx
    out = 6.0 * phi.copy()
    ii = np.arange(nx + 1)
    jj = np.arange(ny + 1)
    out -= phi[:, :, _mirror(ii - 1, nx)] + phi[:, :, _mirror(ii + 1, nx)]
    out -= phi[:, _mirror(jj - 1, ny), :] + phi[:, _mirror(jj + 1, ny), :]
    up = np.zeros_like(phi); up[:-1] = phi[1:]
    dn = np.zeros_like(phi); dn[1:] = phi[:-1]
    out -= up + dn
    return out / dx ** 2


def _assemble(grid):
    """Sparse matrix dx^2 * A over all nodes (rows of Dirichlet nodes are identity)."""
    nx, ny, nz, dx = grid.nx, grid.ny, grid.nz, grid.dx
    dmask = grid.dirichlet_mask().ravel()
    n = grid.nnode
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    k, j, i = k.ravel(), j.ravel(), i.ravel()
    row = np.arange(n)
    free = ~dmask
    rows = [row[dmask]]
    cols = [row[dmask]]
    vals = [np.ones(dmask.sum())]
    # free rows are stored multiplied by dx^2 (entries of order one next to identity rows)
    rows.append(row[free]); cols.append(row[free]); vals.append(np.full(free.sum(), 6.0))
    for (di, dj, dk) in ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)):
        ni = _mirror(i + di, nx)
        nj = _mirror(j + dj, ny)
        nk = k + dk
        ok = free & (nk >= 0) & (nk <= nz)
        col = grid.node_index(ni[ok], nj[ok], nk[ok])
        rows.append(row[ok]); cols.append(col); vals.append(np.full(ok.sum(), -1.0))
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return A, dmask


def rhs_from_charge(grid, Q, w_min, frac_bits=10):
    """rho_n/eps0 from the fixed-point node charge Q (units e*w_min*2^-3F), eq:poi."""
    unit = C.E_CHARGE * w_min * 2.0 ** (-3 * frac_bits)
    return Q.astype(np.float64) * unit / node_volume(grid) / C.EPS0


def solve_poisson(grid, V0, f=None, rtol=1e-13):
    """Solve A phi = f on free nodes with phi fixed on Dirichlet nodes (conjugate gradients)."""
    A, dmask = _assemble(grid)
    n = grid.nnode
    b = np.zeros(n) if f is None else np.asarray(f, dtype=np.float64).ravel() * grid.dx ** 2
    phid = np.where(dmask, grid.dirichlet_values(V0).ravel(), 0.0)
    free = ~dmask
    scale = (node_volume(grid).ravel() / grid.dx ** 3)[free]
    Aff = sp.diags(scale) @ A[free][:, free]
    rhs = scale * (b[free] - A[free] @ phid)
    x, info = spla.cg(Aff.tocsr(), rhs, rtol=rtol, atol=0.0, maxiter=20000)
    if info != 0:
        raise RuntimeError("oracle CG did not converge")
    phi = phid.copy()
    phi[free] = x
    return phi.reshape(grid.nz + 1, grid.ny + 1, grid.nx + 1)


def relative_residual(grid, phi, f, V0):
    """||f - A phi||_2 / ||f_lifted||_2 over free nodes, Dirichlet lifting included in f."""
    dmask = grid.dirichlet_mask()
    r = np.asarray(f, dtype=np.float64) - apply_operator(grid, phi)
    phid = np.where(dmask, grid.dirichlet_values(V0), 0.0)
    lifted = np.asarray(f, dtype=np.float64) - apply_operator(grid, phid)
    num = np.sqrt(np.sum(r[~dmask] ** 2))
    den = np.sqrt(np.sum(lifted[~dmask] ** 2))
    return num / den


def efield(grid, phi):
    """Node field E = -grad(phi) as float32 (nz+1, ny+1, nx+1, 3).

    Central differences phi[n-1] - phi[n+1], taken in FP64 and rounded to f32, times
    f32(1/(2 dx)) in f32; mirror images across the lateral boundaries (E_x = 0 on x=0 and
    x=nx); one-sided differences times f32(1/dx) on the z=0 and z=nz planes.  The paper leaves
    the field arithmetic open (Sec. 2.2 defers to the FEM code it cites); this reading keeps E
    within ~1.2e-7 relative of the exact difference quotient and fixes the op order, because
    the kick decisions that follow use the kernel's precision."""
    nx, ny, nz, dx = grid.nx, grid.ny, grid.nz, grid.dx
    inv2 = np.float32(1.0 / (2.0 * dx))
    inv1 = np.float32(1.0 / dx)
    ii = np.arange(nx + 1)
    jj = np.arange(ny + 1)
    f32 = np.float32
    E = np.zeros((nz + 1, ny + 1, nx + 1, 3), dtype=np.float32)
    E[..., 0] = (phi[:, :, _mirror(ii - 1, nx)] - phi[:, :, _mirror(ii + 1, nx)]).astype(f32) * inv2
    E[..., 1] = (phi[:, _mirror(jj - 1, ny), :] - phi[:, _mirror(jj + 1, ny), :]).astype(f32) * inv2
    E[1:-1, ..., 2] = (phi[:-2] - phi[2:]).astype(f32) * inv2
    E[0, ..., 2] = (phi[0] - phi[1]).astype(f32) * inv1
    E[-1, ..., 2] = (phi[-2] - phi[-1]).astype(f32) * inv1
    return E


def face_field(grid, phi):
    """Local surface field F_f [V/m] of every exposed face: mean over the face's 4 corner
    nodes of (phi one dx outward along the normal - phi at the corner) / dx."""
    F = np.zeros(grid.nface)
    for f in range(grid.nface):
        axis, sign, plane, ijk = grid.face_geometry(f)
        t = [a for a in range(3) if a != axis]
        acc = 0.0
        for a in (0, 1):
            for b in (0, 1):
                c = [0, 0, 0]
                c[axis] = plane
                c[t[0]] = ijk[t[0]] + a
                c[t[1]] = ijk[t[1]] + b
                o = list(c)
                o[axis] = plane + sign
                acc += phi[o[2], o[1], o[0]] - phi[c[2], c[1], c[0]]
        F[f] = acc / 4.0 / grid.dx
    return F


def calibrate_V0(grid, apex_field):
    """V0 such that the mean face field over the apex faces equals apex_field (Laplace, V0=1)."""
    phi1 = solve_poisson(grid, 1.0)
    F1 = face_field(grid, phi1)[grid.apex_faces()].mean()
    return apex_field / F1
