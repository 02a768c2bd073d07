"""Implicit time marching of the DG residual (Sec. II.B.3), FP64.  Test
infrastructure only.

The paper integrates eq. byparts with singly diagonally implicit Runge-Kutta
(SDIRK) methods: a four-stage fourth-order scheme for the Couette order study
and the one-stage first-order scheme (backward Euler, the backward difference
method) for the cavities; every stage is linearised by Newton's method.  The
paper prints no tableau for its fourth-order scheme, so two published
fourth-order SDIRK tableaux stand in for it (see TABLEAUX).

For stage i of a step from u_n with step dt, the stage value solves

    Y_i = u_n + dt sum_{j<i} a_ij k_j + dt gamma R(Y_i),

k_i = (Y_i - base_i) / (dt gamma) (equal to R(Y_i) at convergence), and
u_{n+1} = u_n + dt sum_i b_i k_i.  Here each stage equation is solved by
Newton's method with a dense finite-difference Jacobian of R (small problems
only), which is a plainly different solver from the library's matrix-free
Newton-GMRES.
"""
import numpy as np
from scipy.linalg import lu_factor, lu_solve


def _crouzeix_3_4():
    # Crouzeix (1975), Norsett: 3 stages, order 4, A-stable
    g = 0.5 + np.cos(np.pi / 18.0) / np.sqrt(3.0)
    d = 1.0 / (6.0 * (2.0 * g - 1.0) ** 2)
    A = np.array([[g, 0.0, 0.0],
                  [0.5 - g, g, 0.0],
                  [2.0 * g, 1.0 - 4.0 * g, g]])
    return A, np.array([d, 1.0 - 2.0 * d, d])


def _hairer_wanner_5_4():
    # Hairer & Wanner, Solving ODEs II, Sec. IV.6: 5 stages, order 4,
    # L-stable, gamma = 1/4, stiffly accurate
    A = np.array([[1 / 4, 0, 0, 0, 0],
                  [1 / 2, 1 / 4, 0, 0, 0],
                  [17 / 50, -1 / 25, 1 / 4, 0, 0],
                  [371 / 1360, -137 / 2720, 15 / 544, 1 / 4, 0],
                  [25 / 24, -49 / 48, 125 / 16, -85 / 12, 1 / 4]], dtype=np.float64)
    return A, A[-1].copy()


TABLEAUX = {
    "be": (np.array([[1.0]]), np.array([1.0])),
    "sdirk3o4": _crouzeix_3_4(),
    "sdirk5o4": _hairer_wanner_5_4(),
}


def dense_jacobian(problem, f, h=1e-7):
    """dR/df at f by one-sided finite differences, [n, n]."""
    shape = f.shape
    x = f.ravel()
    r0 = problem.rhs(x.reshape(shape)).ravel()
    J = np.empty((x.size, x.size))
    step = h * max(1.0, np.abs(x).max())
    for j in range(x.size):
        v = x.copy()
        v[j] += step
        J[:, j] = (problem.rhs(v.reshape(shape)).ravel() - r0) / step
    return J


def sdirk_step(problem, f, dt, scheme="be", tol=1e-13, max_iter=30, J=None):
    """One SDIRK step of the DG system df/dt = R(f) from f [K, Np, Q].

    Newton with the Jacobian taken once at f (simplified Newton); R is
    affine in f apart from the equilibrium in the collision term, so it
    converges in a few iterations.  Returns (f_new, stats)."""
    A, b = TABLEAUX[scheme] if isinstance(scheme, str) else scheme
    s = len(b)
    gamma = A[0, 0]
    shape = f.shape
    u0 = f.ravel()
    n = u0.size
    if J is None:
        J = dense_jacobian(problem, f)
    lu = lu_factor(np.eye(n) - dt * gamma * J)
    R = lambda v: problem.rhs(v.reshape(shape)).ravel()
    ks = []
    iters = 0
    Y = u0.copy()
    for i in range(s):
        base = u0 + dt * sum(A[i, j] * ks[j] for j in range(i)) if i else u0.copy()
        for _ in range(max_iter):
            G = Y - base - dt * gamma * R(Y)
            if np.abs(G).max() < tol:
                break
            Y = Y - lu_solve(lu, G)
            iters += 1
        ks.append((Y - base) / (dt * gamma))
    u1 = u0 + dt * sum(b[i] * ks[i] for i in range(s))
    return u1.reshape(shape), {"newton_iters": iters}


def march(problem, f, dt, nsteps, scheme="be", **kw):
    """nsteps SDIRK steps with the Jacobian taken once at the initial state."""
    J = dense_jacobian(problem, f)
    for _ in range(nsteps):
        f, _ = sdirk_step(problem, f, dt, scheme, J=J, **kw)
    return f
