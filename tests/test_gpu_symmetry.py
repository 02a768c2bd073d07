"""The CUDA path's lid-driven cavity commutes with the square's reflections.

The discrete method of Sec. II.B is equivariant under an isometry of the
square that maps the mesh to a mesh of the same kind, acting on positions,
velocities and wall velocities together (the property and its oracle pin are
in test_oracle_cavity_symmetry.py).  Here the original cavity runs on the
library's structured split-square mesh and its image on the library's
triangle-list path (the reflection x -> 1 - x turns the diagonals the other
way); the image of the original run must equal the image run.  This checks
the CUDA path against a property that holds at any size, so it runs up to the
full benchmark mesh, where the oracle itself would be slow."""
import numpy as np
import pytest

from tests import cases
from tests import test_oracle_cavity_symmetry as tsym

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def run_pair(n, p, vs, prec, iso, nsteps, kn=1.0):
    A, b = tsym.MIRROR_X if iso == "mirror_x" else tsym.DIAGONAL
    c = cases.cavity(n, n, p, velset=vs, kn=kn)
    vert, tri = tsym.square_triangles(n)
    vert2 = vert @ A.T + b
    tri2 = tri[:, ::-1].copy() if np.linalg.det(A) < 0 else tri.copy()
    wall2 = np.zeros((4, 2))
    for s in range(4):
        n2 = A @ tsym.dg.SIDE_NORMAL[s]
        wall2[int(np.argmin(np.abs(tsym.dg.SIDE_NORMAL - n2).sum(axis=1)))] = A @ np.asarray(c["wall_u"][s], float)
    c2 = dict(c, mesh=(vert2, tri2), wall_u=tuple(map(tuple, wall2)))
    pr, pr2 = cases.oracle_problem(c), cases.oracle_problem(c2)
    j = tsym.velocity_image(pr, A)
    n2 = tsym.node_image(pr, pr2, A, b)
    kk = np.arange(pr.K)[:, None, None]
    f0 = cases.initial_state(pr, amp=0.05, seed=7)
    f0_2 = np.empty_like(f0)
    f0_2[kk, n2[:, :, None], j[None, None, :]] = f0
    out = []
    for case, state in ((c, f0), (c2, f0_2)):
        s = cases.solver(case, prec)
        s.set_state(state)
        s.step(nsteps)
        out.append(s.state())
        s.close()
    f, f2 = out
    img = f2[kk, n2[:, :, None], j[None, None, :]]
    assert np.abs(f - f0).max() > 1e-4              # the flow moved away from the initial state
    return pr, cases.rel_max_err(img, f)


@pytest.mark.parametrize("iso", ["mirror_x", "diagonal"])
def test_cuda_cavity_reflections_fp64(iso):
    pr, err = run_pair(12, 3, ("gh", 4), "fp64", iso, 3)
    assert err < 1e-12, err


@pytest.mark.parametrize("iso", ["mirror_x", "diagonal"])
def test_cuda_cavity_reflections_fp32_full_benchmark_mesh(iso):
    # the benchmark's cavity (64 x 64 x 2, p = 4, NC 16 x 16) in the default
    # FP32 form: each run rounds on its own (node and velocity orders differ),
    # so the two may differ by twice the FP32 bound each meets against the oracle
    pr, err = run_pair(64, 4, ("nc", 16), "fp32", iso, 2)
    assert err < 2 * (4.0 * pr.Np * U32 * np.sqrt(10) + U32), err
