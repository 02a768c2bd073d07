"""Triangulations and face connectivity (Sec. II.B.1; Sec. III.A builds its
grids by splitting Cartesian squares into two triangles, Sec. III.B runs the
cavity on unstructured meshes).  Test infrastructure only.

Element numbering (a definition shared, as a convention, with the CUDA
library): square (ix, iy) of an Nx x Ny grid on [0, Lx] x [0, Ly] has corners
A = (ix, iy), B = (ix+1, iy), C = (ix+1, iy+1), D = (ix, iy+1) (in cell
units) and is split along the diagonal A-C.  Element k = 2*(iy*Nx + ix) + t
with t = 0 -> (A, B, C) and t = 1 -> (A, C, D); both counter-clockwise.
Face f of an element joins its vertices f and (f+1) mod 3.

Boundary sides: 0 -> y = 0, 1 -> x = Lx, 2 -> y = Ly, 3 -> x = 0.
"""
import numpy as np


def structured_mesh(Nx, Ny, Lx=1.0, Ly=1.0):
    """Vertex coordinates vx, vy of shape [K, 3]."""
    hx, hy = Lx / Nx, Ly / Ny
    K = 2 * Nx * Ny
    vx = np.zeros((K, 3))
    vy = np.zeros((K, 3))
    for iy in range(Ny):
        for ix in range(Nx):
            A = (ix * hx, iy * hy)
            B = ((ix + 1) * hx, iy * hy)
            C = ((ix + 1) * hx, (iy + 1) * hy)
            D = (ix * hx, (iy + 1) * hy)
            base = 2 * (iy * Nx + ix)
            for t, tri in enumerate(((A, B, C), (A, C, D))):
                for v in range(3):
                    vx[base + t, v] = tri[v][0]
                    vy[base + t, v] = tri[v][1]
    return vx, vy


def element_vertices(vert_xy, tri):
    """Vertex coordinates vx, vy [K, 3] of a triangulation given as vertices
    [nv, 2] and counter-clockwise triangles [K, 3] (vertex indices); the faces
    of element k then join its vertices f and (f+1) mod 3 as above."""
    v = np.asarray(vert_xy, dtype=np.float64)
    t = np.asarray(tri, dtype=np.int64)
    return v[t, 0].copy(), v[t, 1].copy()


def boundary_side(x0, y0, x1, y1, Lx, Ly, tol=1e-12):
    """Side id of a face with end points (x0,y0)-(x1,y1), or -1 if interior."""
    if abs(y0) < tol and abs(y1) < tol:
        return 0
    if abs(x0 - Lx) < tol and abs(x1 - Lx) < tol:
        return 1
    if abs(y0 - Ly) < tol and abs(y1 - Ly) < tol:
        return 2
    if abs(x0) < tol and abs(x1) < tol:
        return 3
    return -1


def connectivity(vx, vy, Lx, Ly, periodic_x, periodic_y):
    """Face neighbours found by matching face midpoints.

    Returns (nbr_elem, nbr_face, side), each [K, 3] int.  For a wall face
    nbr_elem = nbr_face = -1 and side holds the boundary side; for a
    periodic boundary face the neighbour is the element across the opposite
    side; side = -1 for interior faces.
    """
    K = vx.shape[0]
    key = {}

    def mkey(x, y):
        return (round(x * 1e9), round(y * 1e9))

    mids = np.zeros((K, 3, 2))
    for k in range(K):
        for f in range(3):
            a, b = f, (f + 1) % 3
            mx = 0.5 * (vx[k, a] + vx[k, b])
            my = 0.5 * (vy[k, a] + vy[k, b])
            mids[k, f] = (mx, my)
            key.setdefault(mkey(mx, my), []).append((k, f))
    nbr_elem = -np.ones((K, 3), dtype=np.int64)
    nbr_face = -np.ones((K, 3), dtype=np.int64)
    side = -np.ones((K, 3), dtype=np.int64)
    for k in range(K):
        for f in range(3):
            a, b = f, (f + 1) % 3
            s = boundary_side(vx[k, a], vy[k, a], vx[k, b], vy[k, b], Lx, Ly)
            side[k, f] = s
            mx, my = mids[k, f]
            if s < 0:
                cands = [c for c in key[mkey(mx, my)] if c != (k, f)]
            elif s in (1, 3) and periodic_x:
                cands = key[mkey(0.0 if s == 1 else Lx, my)]
            elif s in (0, 2) and periodic_y:
                cands = key[mkey(mx, Ly if s == 0 else 0.0)]
            else:
                cands = []
            if s >= 0 and cands == []:
                continue
            assert len(cands) == 1, (k, f, cands)
            nbr_elem[k, f], nbr_face[k, f] = cands[0]
    return nbr_elem, nbr_face, side


def inscribed_radius(vx, vy):
    """Inscribed radius 2*area/perimeter of every element, [K]."""
    la = np.hypot(vx[:, 1] - vx[:, 0], vy[:, 1] - vy[:, 0])
    lb = np.hypot(vx[:, 2] - vx[:, 1], vy[:, 2] - vy[:, 1])
    lc = np.hypot(vx[:, 0] - vx[:, 2], vy[:, 0] - vy[:, 2])
    area = 0.5 * np.abs((vx[:, 1] - vx[:, 0]) * (vy[:, 2] - vy[:, 0])
                        - (vx[:, 2] - vx[:, 0]) * (vy[:, 1] - vy[:, 0]))
    return 2.0 * area / (la + lb + lc)
