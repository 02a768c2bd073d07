"""Pins of the oracle's nodal DG operators and geometry (Sec. II.B.1)."""
from math import factorial

import numpy as np
import pytest

from oracle import mesh, ops


@pytest.mark.parametrize("p", range(0, 7))
def test_derivatives_exact_on_polynomials(p):
    o = ops.RefOps(p)
    r, s = o.r, o.s
    for a in range(p + 1):
        for b in range(p + 1 - a):
            u = r ** a * s ** b
            dur = a * r ** max(a - 1, 0) * s ** b if a else np.zeros_like(r)
            dus = b * r ** a * s ** max(b - 1, 0) if b else np.zeros_like(r)
            np.testing.assert_allclose(o.Dr @ u, dur, atol=1e-12)
            np.testing.assert_allclose(o.Ds @ u, dus, atol=1e-12)


@pytest.mark.parametrize("p", range(0, 7))
def test_mass_matrix_integrates_products(p):
    # with u = (1+r)/2, v = (1+s)/2:  int_T u^a v^b dr ds = 4 a! b! / (a+b+2)!
    o = ops.RefOps(p)
    u = 0.5 * (1 + o.r)
    v = 0.5 * (1 + o.s)
    assert abs(np.ones(o.Np) @ o.M @ np.ones(o.Np) - 2.0) < 1e-13
    for a in range(p + 1):
        for b in range(p + 1):
            exact = 4.0 * factorial(a) * factorial(b) / factorial(a + b + 2)
            assert abs((u ** a) @ o.M @ (v ** b) - exact) < 1e-13


@pytest.mark.parametrize("p", range(0, 7))
def test_face_mass_integrates_edge_polynomials(p):
    o = ops.RefOps(p)
    Nfp = o.Nfp
    t_of_face = [o.r[o.fmask[0]], o.s[o.fmask[1]], o.s[o.fmask[2]]]
    for f in range(3):
        E = o.Emat[:, f * Nfp:(f + 1) * Nfp]
        # rows outside the face vanish
        off = np.setdiff1d(np.arange(o.Np), o.fmask[f])
        assert np.abs(E[off]).max(initial=0.0) < 1e-13
        t = t_of_face[f]
        for m in range(p + 1):
            g = t ** m if Nfp > 1 else np.ones(1)
            exact = (1 - (-1) ** (m + 1)) / (m + 1)
            if Nfp == 1 and m > 0:
                continue
            assert abs(np.ones(o.Np) @ E @ g - exact) < 1e-13
    np.testing.assert_allclose(o.M @ o.LIFT, o.Emat, atol=1e-12)


def test_nodes_low_order_equispaced_and_edges_gll():
    r, s = ops.nodes(2)
    np.testing.assert_allclose(r, [-1, 0, 1, -1, 0, -1], atol=1e-15)
    np.testing.assert_allclose(s, [-1, -1, -1, 0, 0, 1], atol=1e-15)
    want = {3: [-1, -1 / np.sqrt(5), 1 / np.sqrt(5), 1],
            4: [-1, -np.sqrt(3 / 7), 0, np.sqrt(3 / 7), 1]}
    for p, gll in want.items():
        o = ops.RefOps(p)
        np.testing.assert_allclose(o.r[o.fmask[0]], gll, atol=1e-14)
        np.testing.assert_allclose(o.s[o.fmask[2]], gll, atol=1e-14)
        np.testing.assert_allclose(o.s[o.fmask[1]], gll, atol=1e-14)


@pytest.mark.parametrize("p", range(1, 7))
def test_nodes_symmetric_and_inside(p):
    r, s = ops.nodes(p)
    assert len(r) == (p + 1) * (p + 2) // 2
    pts = set(zip(np.round(r, 10), np.round(s, 10)))
    assert pts == set(zip(np.round(s, 10), np.round(r, 10)))      # r <-> s mirror
    assert np.all(r >= -1 - 1e-14) and np.all(s >= -1 - 1e-14) and np.all(r + s <= 1e-14)


def test_geometry_structured_mesh():
    vx, vy = mesh.structured_mesh(3, 2, 1.0, 1.0)
    g = ops.geometry(vx, vy)
    np.testing.assert_allclose(g["J"], (1 / 3) * (1 / 2) / 4)
    np.testing.assert_allclose(np.hypot(g["nx"], g["ny"]), 1.0)
    # sum_f |face| n_f = 0 for each closed triangle
    np.testing.assert_allclose((2 * g["sJ"] * g["nx"]).sum(1), 0, atol=1e-15)
    np.testing.assert_allclose((2 * g["sJ"] * g["ny"]).sum(1), 0, atol=1e-15)
    # outward: the normal points away from the centroid
    cx, cy = vx.mean(1), vy.mean(1)
    for f in range(3):
        mx = 0.5 * (vx[:, f] + vx[:, (f + 1) % 3])
        my = 0.5 * (vy[:, f] + vy[:, (f + 1) % 3])
        assert np.all((mx - cx) * g["nx"][:, f] + (my - cy) * g["ny"][:, f] > 0)
    rin = mesh.inscribed_radius(vx, vy)
    a, b = 1 / 3, 1 / 2
    np.testing.assert_allclose(rin, a * b / (a + b + np.hypot(a, b)))


def test_connectivity_periodic_and_walls():
    vx, vy = mesh.structured_mesh(3, 3)
    ne, nf, side = mesh.connectivity(vx, vy, 1.0, 1.0, True, False)
    # periodic in x: every face has a neighbour except y walls
    walls = ne < 0
    assert set(side[walls].tolist()) == {0, 2}
    assert walls.sum() == 6
    for k in range(ne.shape[0]):
        for f in range(3):
            if ne[k, f] >= 0:
                assert ne[ne[k, f], nf[k, f]] == k and nf[ne[k, f], nf[k, f]] == f
