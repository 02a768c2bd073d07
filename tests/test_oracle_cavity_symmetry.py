"""The oracle's lid-driven cavity (and Couette flow) pinned by the symmetries
of the square.

The cavity of Sec. III.B has no closed-form solution, but the discrete method
of Sec. II.B commutes with every isometry of the square that maps the mesh to
a mesh of the same kind: the BGK equation is invariant under a rotation or
reflection x -> A x + b acting on positions and velocities together
(e_i -> A e_i permutes a tensor-product velocity set; f^eq of eq. feq depends
only on e.u and u.u), the nodal DG operators on the image triangles are the
images of the original ones (the warp & blend node set is invariant under the
symmetries of the triangle), and the walls of eq. FullBC map to walls whose
velocity is A u_b.  So, with the image of the state as initial state, the
image problem must step to the image of the original solution, up to
rounding.  Two isometries are used:

* the reflection x -> 1 - x: the lid velocity (U, 0) becomes (-U, 0), and the
  split-square mesh becomes one whose diagonals run the other way (handed to
  the oracle as a triangle list);
* the reflection across the diagonal y = x: the lid moves from y = 1 to
  x = 1 with velocity (0, U), and the split-square mesh maps to itself;
* for Couette flow (Sec. III.A), the rotation by pi about the centre: the
  plates change places with their velocities reversed, which is the same
  problem, and the periodic seam maps onto itself.

A mistake that treats x and y, or the two orientations of a face, unequally --
a wrong metric term, a lid-velocity component taken from the wrong axis, a
face-node map that depends on orientation -- breaks one of them; mistakes
that keep the symmetry are left to the other pins."""
import numpy as np
import pytest

from oracle import dg
from tests import cases

CAV = ("diffuse",) * 4


def square_triangles(n):
    """The n x n split-square mesh of the unit square as vertices [nv, 2] and
    counter-clockwise triangles [K, 3] in the oracle's element order."""
    g = np.linspace(0.0, 1.0, n + 1)
    vert = np.array([(x, y) for y in g for x in g])
    vid = lambda ix, iy: iy * (n + 1) + ix
    tri = []
    for iy in range(n):
        for ix in range(n):
            a, b, c, d = vid(ix, iy), vid(ix + 1, iy), vid(ix + 1, iy + 1), vid(ix, iy + 1)
            tri += [(a, b, c), (a, c, d)]
    return vert, np.array(tri)


def image_problem(pr, mesh, A, b, wall_u, bc=CAV, **kw):
    """The problem on the image of `mesh` under x -> A x + b, with every side's
    kind and wall velocity mapped (by A) onto the image of the side; triangles
    of a reflected mesh are reversed so that they stay counter-clockwise."""
    vert, tri = mesh
    vert2 = vert @ A.T + b
    tri2 = tri[:, ::-1].copy() if np.linalg.det(A) < 0 else tri.copy()
    wall2 = np.zeros((4, 2))
    bc2 = [None] * 4
    for s in range(4):
        n2 = A @ dg.SIDE_NORMAL[s]
        s2 = int(np.argmin(np.abs(dg.SIDE_NORMAL - n2).sum(axis=1)))
        assert np.allclose(dg.SIDE_NORMAL[s2], n2)
        wall2[s2] = A @ np.asarray(wall_u[s], dtype=float)
        bc2[s2] = bc[s]
    return dg.Problem(0, 0, pr.p, bc=tuple(bc2), wall_u=tuple(map(tuple, wall2)), mesh=(vert2, tri2),
                      dt=pr.dt, **kw)


def velocity_image(pr, A):
    """j[i]: index of the velocity A e_i (the set is mapped onto itself)."""
    e = np.stack([pr.ex, pr.ey], axis=1)
    e2 = e @ A.T
    j = np.array([int(np.argmin(np.abs(e - v).sum(axis=1))) for v in e2])
    assert np.abs(e[j] - e2).max() < 1e-12 and np.abs(pr.w[j] - pr.w).max() < 1e-15
    return j


def node_image(pr, pr2, A, b):
    """n2[k, n]: the node of element k of the image problem (the image of
    triangle k) at the image of node n of element k."""
    n2 = np.empty((pr.K, pr.Np), dtype=np.int64)
    for k in range(pr.K):
        x = np.stack([pr.x[k], pr.y[k]], axis=1) @ A.T + b
        x2 = np.stack([pr2.x[k], pr2.y[k]], axis=1)
        for n in range(pr.Np):
            d = np.abs(x2 - x[n]).sum(axis=1)
            n2[k, n] = int(np.argmin(d))
            assert d[n2[k, n]] < 1e-12
        assert len(np.unique(n2[k])) == pr.Np
    return n2


MIRROR_X = (np.array([[-1.0, 0.0], [0.0, 1.0]]), np.array([1.0, 0.0]))
DIAGONAL = (np.array([[0.0, 1.0], [1.0, 0.0]]), np.array([0.0, 0.0]))
ROTATE_PI = (np.array([[-1.0, 0.0], [0.0, -1.0]]), np.array([1.0, 1.0]))
COUETTE_BC = ("diffuse", "periodic", "diffuse", "periodic")


def check_isometry(A, b, p=2, velset=("gh", 4), eq_order=2, kn=1.0, lid=0.1, n=3, nsteps=2, couette=False):
    """Relative max difference between the original run and the image of the
    image run.  The cavity has its lid (lid, 0) at y = 1; the Couette case
    (periodic in x) has walls (-lid, 0) at y = 0 and (lid, 0) at y = 1."""
    mesh = square_triangles(n)
    if couette:
        bc, wall_u = COUETTE_BC, ((-lid, 0.0), (0.0, 0.0), (lid, 0.0), (0.0, 0.0))
    else:
        bc, wall_u = CAV, ((0.0, 0.0), (0.0, 0.0), (lid, 0.0), (0.0, 0.0))
    kw = dict(velset=velset, eq_order=eq_order, kn=kn)
    pr = dg.Problem(0, 0, p, bc=bc, wall_u=wall_u, mesh=mesh, **kw)
    pr2 = image_problem(pr, mesh, A, b, wall_u, bc=bc, **kw)
    j = velocity_image(pr, A)
    n2 = node_image(pr, pr2, A, b)
    kk = np.arange(pr.K)[:, None, None]
    f0 = cases.initial_state(pr, amp=0.05, seed=7)
    f0_2 = np.empty_like(f0)
    f0_2[kk, n2[:, :, None], j[None, None, :]] = f0
    f = pr.run(f0, nsteps)
    f2 = pr2.run(f0_2, nsteps)
    img = f2[kk, n2[:, :, None], j[None, None, :]]
    # the flow is not symmetric by itself, so the check is not vacuous
    assert np.abs(f - f0).max() > 1e-4
    return float(np.abs(img - f).max() / np.abs(f).max())


@pytest.mark.parametrize("iso", ["mirror_x", "diagonal"])
@pytest.mark.parametrize("p,velset,eq_order", [(2, ("gh", 4), 2), (3, ("nc", 6), 3), (1, ("gh", 5), 2)])
def test_cavity_commutes_with_square_isometries(iso, p, velset, eq_order):
    A, b = MIRROR_X if iso == "mirror_x" else DIAGONAL
    assert check_isometry(A, b, p=p, velset=velset, eq_order=eq_order) < 1e-13


@pytest.mark.parametrize("p,velset", [(2, ("gh", 4)), (3, ("nc", 6))])
def test_couette_commutes_with_rotation_by_pi(p, velset):
    # the point reflection about the centre maps the plates onto each other
    # with their velocities reversed, i.e. the Couette problem onto itself,
    # and carries the periodic seam x = 0 ~ x = 1 onto itself
    assert check_isometry(*ROTATE_PI, p=p, velset=velset, couette=True, n=4) < 1e-13


def test_diagonal_reflection_maps_the_split_square_mesh_to_itself():
    # the element set of the image mesh is the original one (permuted), so the
    # diagonal check runs the cavity on the very mesh of the benchmark cases
    vert, tri = square_triangles(4)
    A, b = DIAGONAL
    cent = lambda v: sorted(map(tuple, np.round(v[tri].mean(axis=1), 12)))
    assert cent(vert) == cent(vert @ A.T + b)


def pins():
    """The pins as one call, for the planted-mistake tests."""
    for iso in (MIRROR_X, DIAGONAL):
        assert check_isometry(*iso) < 1e-13
    assert check_isometry(*ROTATE_PI, couette=True, n=4) < 1e-13
