"""The oracle on unstructured triangulations (Sec. III.B runs the cavity on
unstructured meshes; the paper's mesh file is not available, so seeded
jittered meshes with random diagonals, rotated vertex lists and shuffled
element order stand in for it), pinned to what the method fixes on any
conforming mesh:

* a uniform equilibrium on a fully periodic mesh is steady (free stream);
* diffuse walls conserve mass: sum_k J_k 1^T M sum_i rhs_i = 0;
* with the collision off, each velocity is translated exactly, and the
  discrete solution converges to g(x - e t) at order about p + 1;
* a structured split-square mesh handed over as a vertex / triangle list
  gives the structured residual bit for bit up to face order;

and the C library's host-side mesh set-up (connectivity codes and node
coordinates) agrees with the oracle's independent construction."""
import numpy as np
import pytest

from oracle import dg
from paper_2012_13487_gb300 import inputs

PER = ("periodic",) * 4
CAV = ("diffuse",) * 4


def _mesh(nx, ny, seed=11, **kw):
    return inputs.unstructured_square(nx, ny, seed, **kw)


def test_generator_mesh_is_conforming_and_counter_clockwise():
    v, t = _mesh(5, 4)
    X = v[t]
    area2 = (X[:, 1, 0] - X[:, 0, 0]) * (X[:, 2, 1] - X[:, 0, 1]) - (X[:, 2, 0] - X[:, 0, 0]) * (X[:, 1, 1] - X[:, 0, 1])
    assert np.all(area2 > 0)
    assert abs(area2.sum() / 2 - 1.0) < 1e-14           # the triangles tile the unit square
    edges = {}
    for k in range(len(t)):
        for f in range(3):
            a, b = t[k, f], t[k, (f + 1) % 3]
            edges.setdefault((min(a, b), max(a, b)), []).append((a, b))
    for (a, b), uses in edges.items():
        assert len(uses) in (1, 2)
        if len(uses) == 2:
            assert uses[0] == uses[1][::-1]              # traversed in opposite directions


@pytest.mark.parametrize("p", [1, 3])
def test_free_stream_on_periodic_unstructured_mesh(p):
    pr = dg.Problem(0, 0, p, velset=("gh", 4), bc=PER, wall_u=((0, 0),) * 4, mesh=_mesh(4, 5))
    f = pr.equilibrium_state(1.1, 0.07, -0.03)
    assert np.abs(pr.rhs(f)).max() < 1e-13


def test_rest_state_with_resting_walls_is_steady_unstructured():
    pr = dg.Problem(0, 0, 2, velset=("nc", 6), bc=CAV, wall_u=((0, 0),) * 4, mesh=_mesh(4, 4, seed=3))
    assert np.abs(pr.rhs(pr.equilibrium_state())).max() < 1e-13


def test_diffuse_walls_conserve_mass_unstructured():
    pr = dg.Problem(0, 0, 3, velset=("gh", 4), bc=CAV, wall_u=((0, 0), (0, 0), (0.1, 0), (0, 0)),
                    mesh=_mesh(4, 3, seed=5))
    f = pr.equilibrium_state(1.0, 0.0, 0.0, 1e-2, inputs.perturbation(3, pr.K, pr.Np, pr.Q))
    r = pr.rhs(f)
    colsum = pr.ops.M.sum(axis=0)
    dmass = np.sum(pr.geo["J"][:, None] * colsum[None, :] * r.sum(axis=-1))
    scale = np.sum(pr.geo["J"][:, None] * colsum[None, :] * np.abs(r).sum(axis=-1))
    assert abs(dmass) < 1e-14 * scale


def test_structured_mesh_as_triangle_list_gives_the_same_residual():
    nx, ny = 3, 2
    pr_s = dg.Problem(nx, ny, 2, velset=("gh", 4), bc=("diffuse", "periodic", "diffuse", "periodic"))
    # the same mesh written as a vertex list and triangles (A, B, C), (A, C, D)
    vert = np.array([(ix / nx, iy / ny) for iy in range(ny + 1) for ix in range(nx + 1)])
    tri = []
    for iy in range(ny):
        for ix in range(nx):
            a = iy * (nx + 1) + ix
            tri += [(a, a + 1, a + nx + 2), (a, a + nx + 2, a + nx + 1)]
    pr_u = dg.Problem(0, 0, 2, velset=("gh", 4), bc=("diffuse", "periodic", "diffuse", "periodic"),
                      mesh=(vert, np.array(tri)))
    f = pr_s.equilibrium_state(1.0, 0.0, 0.0, 1e-2, inputs.perturbation(9, pr_s.K, pr_s.Np, pr_s.Q))
    assert np.abs(pr_u.rhs(f) - pr_s.rhs(f)).max() < 1e-14


def test_advection_order_on_unstructured_meshes():
    def g(x, y):
        return 1.0 + 0.1 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)

    T = 0.05
    errs = []
    for N in (8, 16):
        pr = dg.Problem(0, 0, 2, velset=("gh", 2), bc=PER, wall_u=((0, 0),) * 4, collision=False, cfl=0.25,
                        mesh=_mesh(N, N, seed=N, shuffle=False))
        nsteps = int(np.ceil(T / pr.dt))
        pr.dt = T / nsteps
        f = pr.w[None, None, :] * g(pr.x, pr.y)[:, :, None]
        f = pr.run(f, nsteps)
        exact = pr.w[None, None, :] * g(pr.x[:, :, None] - pr.ex * T, pr.y[:, :, None] - pr.ey * T)
        errs.append(np.abs(f - exact).max())
    rate = np.log2(errs[0] / errs[1])
    assert rate > 2.5, (errs, rate)


def test_library_connectivity_and_nodes_match_the_oracle():
    from paper_2012_13487_gb300 import fedbm as fb
    v, t = _mesh(5, 4, seed=21)
    for bc, obc in (((fb.BC_WALL_DIFFUSE,) * 4, CAV), ((fb.BC_PERIODIC,) * 4, PER),
                    ((fb.BC_WALL_DIFFUSE, fb.BC_PERIODIC, fb.BC_WALL_DIFFUSE, fb.BC_PERIODIC),
                     ("diffuse", "periodic", "diffuse", "periodic"))):
        md = fb.unstructured_mesh_desc(v, t, 3, bc=bc)
        nbr = fb.fedbm_mesh_connectivity(md)
        pr = dg.Problem(0, 0, 3, velset=("gh", 4), bc=obc, wall_u=((0, 0),) * 4, mesh=(v, t))
        for k in range(pr.K):
            for f in range(3):
                code = nbr[k, f]
                if pr.nbr_elem[k, f] < 0:
                    assert code == -(pr.side[k, f] + 1)
                    continue
                assert code >= 0
                assert code >> 3 == pr.nbr_elem[k, f] and (code >> 1) & 3 == pr.nbr_face[k, f]
                # orientation flag: the neighbour's face nodes in opposite order
                fm, fmn = pr.ops.fmask[f], pr.ops.fmask[(code >> 1) & 3]
                order = [int(np.nonzero(fmn == n)[0][0]) for n in pr.mapn[k, f]]
                assert order == (list(range(pr.Nfp))[::-1] if code & 1 else list(range(pr.Nfp)))
        x, y, _ = fb.fedbm_mesh_nodes(md)
        assert np.abs(x - pr.x).max() < 1e-14 and np.abs(y - pr.y).max() < 1e-14


def test_library_rejects_bad_triangulations():
    from paper_2012_13487_gb300 import fedbm as fb
    v, t = _mesh(3, 3, seed=2)
    bad = t.copy()
    bad[4] = bad[4][::-1]                       # clockwise
    with pytest.raises(fb.FedbmError):
        fb.fedbm_mesh_connectivity(fb.unstructured_mesh_desc(v, bad, 2))
    bad = t.copy()
    bad[0, 0] = len(v)                          # index out of range
    with pytest.raises(fb.FedbmError):
        fb.fedbm_mesh_connectivity(fb.unstructured_mesh_desc(v, bad, 2))
    with pytest.raises(fb.FedbmError):          # a hole: boundary edges inside the square
        fb.fedbm_mesh_connectivity(fb.unstructured_mesh_desc(v, t[1:], 2))
    w = v.copy()
    w[w[:, 0] == 1.0, 1] += 1e-3                # right side moved: periodic pairing fails
    w[w[:, 1] > 1.0, 1] = 1.0
    with pytest.raises(fb.FedbmError):
        fb.fedbm_mesh_connectivity(fb.unstructured_mesh_desc(w, t, 2, bc=(fb.BC_PERIODIC,) * 4))
