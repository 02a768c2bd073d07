"""Discrete velocity sets (Sec. II.A.2-3, Table 1).  Test infrastructure only.

Velocities are in units of sqrt(RT) (theta = RT = c_s^2 = 1).  2-D sets are
tensor products of a 1-D rule with index i = ix * n + iy, so that
e_x[i] = x[ix], e_y[i] = x[iy], w[i] = w1[ix] * w1[iy].
"""
import numpy as np
from numpy.polynomial.hermite_e import hermegauss


def gauss_hermite_1d(n):
    """n-point probabilists' Gauss-Hermite rule with unit total weight.

    Weight function exp(-x^2/2)/sqrt(2 pi); exact for polynomials of degree
    2n-1 (Table 1 lists D1Q4/Q5/Q6 of orders 7/9/11).  NumPy's ``hermegauss``
    is used as the library primitive; it integrates exp(-x^2/2), so the
    weights are divided by sqrt(2 pi).
    """
    x, w = hermegauss(n)
    return np.asarray(x, dtype=np.float64), np.asarray(w, dtype=np.float64) / np.sqrt(2.0 * np.pi)


def newton_cotes_1d(n, extent=4.0, scale=1.0):
    """Equispaced ("Newton-Cotes") 1-D velocity rule (Sec. III.B).

    Nodes x_j are n equispaced points on [-extent, extent]; the velocities
    are xi_j = scale * x_j in units of sqrt(RT) (scale = 1 for a grid in units
    of sqrt(RT), scale = sqrt(2) for a grid in units of sqrt(2RT)).  Weights:
    composite trapezoid weights in xi times the Maxwellian density
    exp(-xi^2/2)/sqrt(2 pi), then multiplied by (a + b xi^2 + c xi^4) with
    (a, b, c) solved so that the moments of order 0, 2 and 4 equal those of
    the Maxwellian (1, 1, 3).  Odd moments vanish by symmetry.  The paper
    fixes only the node grid and positivity of the weights; the trapezoid
    base rule and the moment correction are this code's reading.
    """
    x = np.linspace(-extent, extent, n)
    xi = scale * x
    h = xi[1] - xi[0]
    trap = np.full(n, h)
    trap[0] = trap[-1] = 0.5 * h
    w = trap * np.exp(-0.5 * xi * xi) / np.sqrt(2.0 * np.pi)
    # moment matrix: row m (moment 2m), column c (correction term xi^(2c))
    A = np.empty((3, 3))
    for m in range(3):
        for c in range(3):
            A[m, c] = np.sum(w * xi ** (2 * m + 2 * c))
    abc = np.linalg.solve(A, np.array([1.0, 1.0, 3.0]))
    w = w * (abc[0] + abc[1] * xi ** 2 + abc[2] * xi ** 4)
    return xi, w


def tensor_2d(x, w):
    """Tensor product of a 1-D rule: returns (ex, ey, w2) with i = ix*n + iy."""
    n = len(x)
    ex = np.repeat(x, n)
    ey = np.tile(x, n)
    w2 = np.outer(w, w).ravel()
    return ex, ey, w2


def velocity_set(kind, n, extent=4.0, nc_scale=1.0):
    """2-D set: kind 'gh' (Gauss-Hermite) or 'nc' (Newton-Cotes)."""
    if kind == "gh":
        x, w = gauss_hermite_1d(n)
    elif kind == "nc":
        x, w = newton_cotes_1d(n, extent, nc_scale)
    else:
        raise ValueError(kind)
    return tensor_2d(x, w)
