"""Pins of the oracle's SDIRK time marching (Sec. II.B.3):

* the tableaux satisfy the Runge-Kutta order conditions (Butcher) of their
  stated order -- order 1 for backward Euler, all eight conditions of order 4
  for the two fourth-order schemes -- and are singly diagonally implicit;
* on the DG system itself the observed temporal order is 1 and 4, measured
  against an independent integrator (the explicit LSRK(5,4) at a tiny step);
* every step conserves mass with diffuse walls;
* backward Euler with a large step reaches the steady state R(f) = 0 that the
  steady-state solver of the oracle finds by its own route, and a mistaken
  stage formula (a planted error) destroys the fourth order."""
import numpy as np
import pytest

from oracle import dg, implicit
from paper_2012_13487_gb300 import inputs


def _conditions(A, b):
    c = A.sum(axis=1)
    return {
        (1, "b"): (b.sum(), 1.0),
        (2, "bc"): (b @ c, 0.5),
        (3, "bc2"): (b @ c ** 2, 1 / 3),
        (3, "bAc"): (b @ A @ c, 1 / 6),
        (4, "bc3"): (b @ c ** 3, 1 / 4),
        (4, "bcAc"): (b @ (c * (A @ c)), 1 / 8),
        (4, "bAc2"): (b @ A @ c ** 2, 1 / 12),
        (4, "bAAc"): (b @ A @ A @ c, 1 / 24),
    }


@pytest.mark.parametrize("name,order", [("be", 1), ("sdirk3o4", 4), ("sdirk5o4", 4)])
def test_tableau_order_conditions(name, order):
    A, b = implicit.TABLEAUX[name]
    assert np.allclose(np.triu(A, 1), 0.0)
    assert np.allclose(np.diag(A), A[0, 0]) and A[0, 0] > 0
    for (o, key), (got, want) in _conditions(A, b).items():
        if o <= order:
            assert abs(got - want) < 1e-14, (name, key, got, want)
    if order == 1:
        assert abs(_conditions(A, b)[(2, "bc")][0] - 0.5) > 0.1   # and no more


def _small_problem(**kw):
    return dg.Problem(1, 3, 2, velset=("gh", 3), kn=0.5, wall_u=((-0.1, 0), (0, 0), (0.1, 0), (0, 0)), **kw)


def _relaxed_periodic():
    """Fully periodic 2x2x2 mesh, p = 2, D2Q9, Kn = 0.5, from the local
    equilibrium of smooth density and velocity fields, relaxed for two time
    units with the explicit scheme so that the fast (stiff) transients have
    decayed and the classical orders show at moderate steps."""
    pr = dg.Problem(2, 2, 2, velset=("gh", 3), kn=0.5, bc=("periodic",) * 4, wall_u=((0, 0),) * 4)
    rho = 1 + 0.1 * np.sin(2 * np.pi * pr.x) * np.cos(2 * np.pi * pr.y)
    ux = 0.05 * np.sin(2 * np.pi * pr.y)
    uy = 0.05 * np.cos(2 * np.pi * pr.x)
    f0 = dg.equilibrium(rho, ux, uy, pr.ex, pr.ey, pr.w)
    dt0 = pr.dt
    return pr, pr.run(f0, int(2.0 / dt0)), dt0


def _errors(scheme, pr, f0, dt0, T=0.2, steps=(8, 16)):
    pr.dt = T / int(np.ceil(T / (0.25 * dt0)))     # explicit LSRK(5,4) at a quarter of the CFL step
    ref = pr.run(f0, int(round(T / pr.dt)))
    J = implicit.dense_jacobian(pr, f0)
    errs = []
    for nsteps in steps:
        f = f0
        for _ in range(nsteps):
            f, _ = implicit.sdirk_step(pr, f, T / nsteps, scheme, J=J)
        errs.append(np.abs(f - ref).max())
    return errs


@pytest.mark.parametrize("name,order,tol", [("be", 1, 0.2), ("sdirk3o4", 4, 0.3), ("sdirk5o4", 4, 0.1)])
def test_temporal_order_on_the_dg_system(name, order, tol):
    pr, f0, dt0 = _relaxed_periodic()
    errs = _errors(name, pr, f0, dt0)
    rate = np.log2(errs[0] / errs[1])
    assert abs(rate - order) < tol, (errs, rate)


def test_implicit_steps_conserve_mass_with_diffuse_walls():
    pr = dg.Problem(2, 2, 2, velset=("gh", 3), kn=1.0, bc=("diffuse",) * 4,
                    wall_u=((0, 0), (0, 0), (0.1, 0), (0, 0)))
    f0 = pr.equilibrium_state(1.0, 0.0, 0.0, 1e-2, inputs.perturbation(5, pr.K, pr.Np, pr.Q))
    m0 = pr.mass(f0)
    for name in ("be", "sdirk5o4"):
        f = implicit.march(pr, f0, 0.3, 3, name)
        assert abs(pr.mass(f) - m0) < 1e-12 * m0


def test_backward_euler_large_steps_reach_the_steady_state():
    pr = _small_problem()
    f0 = pr.equilibrium_state()
    fs, res = dg.steady_state(pr, f0)
    f = implicit.march(pr, f0, 50.0, 40, "be")
    assert np.abs(pr.rhs(f)).max() < 1e-11 and res < 1e-11
    # two states with residuals below 1e-11, the slowest decay rate of the
    # linearised problem (~1e-2 here) bounds their distance by ~1e-9
    assert np.abs(f - fs).max() < 5e-9
    assert abs(pr.mass(f) - pr.mass(f0)) < 1e-12       # 40 steps, each solved to 1e-13


def test_a_planted_stage_error_loses_the_order():
    # b weights of the 3-stage scheme permuted: a plausible transcription slip
    A, b = implicit.TABLEAUX["sdirk3o4"]
    pr, f0, dt0 = _relaxed_periodic()
    errs = _errors((A, b[[1, 0, 2]]), pr, f0, dt0)
    assert np.log2(errs[0] / errs[1]) < 2.5
