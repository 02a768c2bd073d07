"""Linearized Couette flow for D2Q16 (Sec. III.A, eq. exact).  Test
infrastructure only.

Two independent routes to the steady x-velocity between plates at y = 0
(speed U_bottom) and y = L (speed U_top):

* ``exact_ux``: the printed closed form, read with two repairs that the
  garbled text needs -- the operator missing between the two bracketed
  terms of Z16 is '+', and the coordinate in the sinh and linear terms is
  measured from the channel centre (eta = y - L/2; the printed "y + 1/2"
  is inconsistent with plates at y = 0 and y = 1).
* ``linearized_steady``: the steady linearized discrete-velocity BGK
  equations in y, e_y phi_i' = -(phi_i - [d_rho + e_i . u]) / tau with
  f_i = w_i (1 + phi_i), solved exactly with a matrix exponential and the
  linearized diffuse-wall conditions of eq. FullBC (zero net mass flux).
  It fixes which tau reading of eq. KnTau the closed form belongs to.
"""
import numpy as np
from scipy.linalg import expm

from . import velset as _velset


def exact_ux(y, kn, u_top, u_bottom, L=1.0):
    """Repaired eq. exact: u_x(y) for D2Q16 at Knudsen number kn."""
    y = np.asarray(y, dtype=np.float64)
    dU = u_top - u_bottom
    U = 0.5 * (u_top + u_bottom)
    mu = np.sqrt(3.0 - np.sqrt(6.0)) + np.sqrt(3.0 + np.sqrt(6.0))
    a = 1.0 / (2.0 * kn)
    theta = 1.0 + 2.0 * kn * ((2.0 * np.cosh(a) + mu * np.sinh(a))
                              / (mu * np.cosh(a) + 2.0 * np.sqrt(3.0) * np.sinh(a)))
    Z = mu / (4.0 * kn) * ((4.0 * kn + mu) * np.cosh(a)
                           + 2.0 * (mu * kn + np.sqrt(3.0)) * np.sinh(a))
    eta = y - 0.5 * L
    return np.sinh(eta / (kn * L)) / Z * dU + (eta / L) / theta * dU + U


def linearized_steady(y, tau, u_top, u_bottom, L=1.0, n1d=4, wall="diffuse"):
    """u_x(y) of the linearized steady discrete-velocity problem (GH n1d^2 set)."""
    ex, ey, w = _velset.tensor_2d(*_velset.gauss_hermite_1d(n1d))
    Q = len(w)
    P = np.outer(np.ones(Q), w) + np.outer(ex, w * ex) + np.outer(ey, w * ey)
    A = -(1.0 / tau) * (np.diag(1.0 / ey) @ (np.eye(Q) - P))
    E1 = expm(A * L)
    H = np.sum(np.where(ey > 0, ey, 0.0) * w)
    rows, rhs = [], []
    # bottom wall (outward normal -y): incoming e_y > 0
    for i in range(Q):
        if ey[i] > 0:
            r = np.zeros(Q)
            r[i] = 1.0
            if wall == "diffuse":
                r -= np.where(ey < 0, -ey, 0.0) * w / H
            rows.append(r)
            rhs.append(ex[i] * u_bottom)
    # top wall (outward normal +y): incoming e_y < 0, phi(L) = E1 phi(0)
    for i in range(Q):
        if ey[i] < 0:
            r = np.zeros(Q)
            r[i] = 1.0
            if wall == "diffuse":
                r -= np.where(ey > 0, ey, 0.0) * w / H
            rows.append(r @ E1)
            rhs.append(ex[i] * u_top)
    phi0, *_ = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)
    y = np.atleast_1d(np.asarray(y, dtype=np.float64))
    out = np.array([np.sum(w * ex * (expm(A * yy) @ phi0)) for yy in y])
    return out
