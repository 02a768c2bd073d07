"""Implicit SDIRK time marching on the GPU (Sec. II.B.3: SDIRK with Newton's
method and GMRES), against the oracle's SDIRK steps, which solve every stage
with a dense finite-difference Jacobian instead of the library's matrix-free
Newton-GMRES; tolerances follow from the solver tolerances requested."""
import numpy as np
import pytest

from oracle import couette, dg, implicit
from tests import cases

pytestmark = pytest.mark.gpu


def _tight(scheme, dt, **kw):
    from paper_2012_13487_gb300 import fedbm as fb
    # the stage equations are solved to |G| <= 1e-12 |G_0| (or 1e-13 absolute,
    # near the FP64 rounding of dt R), so the results agree to ~1e-11 relative
    args = dict(newton_rtol=1e-12, newton_atol=1e-13, newton_max_iter=30, gmres_restart=80,
                gmres_max_iter=2000, gmres_rtol=1e-10)
    args.update(kw)
    return fb.implicit_params(scheme, dt, **args)


def _couette_small():
    return cases.couette(1, 3, 2, velset=("gh", 3), kn=0.5)


@pytest.mark.parametrize("scheme,name", [(0, "be"), (1, "sdirk3o4"), (2, "sdirk5o4")])
def test_implicit_steps_match_oracle_fp64(scheme, name):
    c = _couette_small()
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=2e-2, seed=12)
    dt = 20 * pr.dt                       # well past the explicit CFL limit
    s = cases.solver(c, "fp64")
    s.set_state(f0)
    st = s.implicit_step(_tight(scheme, dt), 2)
    assert st.converged == 1 and st.gmres_iters > 0
    assert abs(s.info.time - 2 * dt) < 1e-15
    f_or = implicit.march(pr, f0, dt, 2, name)
    assert cases.rel_max_err(s.state(), f_or) < 1e-10
    assert abs(s.mass() - pr.mass(f0)) < 1e-12


def test_implicit_fp32_state():
    c = _couette_small()
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=2e-2, seed=13)
    dt = 10 * pr.dt
    s = cases.solver(c, "fp32")
    s.set_state(f0)
    # FP32 residuals: Newton to the FP32 rounding level of G
    st = s.implicit_step(_tight(0, dt, newton_rtol=1e-5, newton_atol=1e-6, gmres_rtol=1e-5), 1)
    assert st.converged == 1
    f_or, _ = implicit.sdirk_step(pr, f0, dt, "be")
    assert cases.rel_max_err(s.state(), f_or) < 2e-6


def test_custom_tableau_equals_backward_euler():
    from paper_2012_13487_gb300 import fedbm as fb
    c = _couette_small()
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=2e-2, seed=14)
    out = []
    for ip in (_tight(0, 0.05), fb.implicit_params(fb.IMPLICIT_CUSTOM, 0.05, newton_rtol=1e-12, newton_atol=1e-13,
                                                   newton_max_iter=30, gmres_restart=80, gmres_max_iter=2000,
                                                   gmres_rtol=1e-10, A=[[1.0]], b=[1.0])):
        s = cases.solver(c, "fp64")
        s.set_state(f0)
        s.implicit_step(ip, 1)
        out.append(s.state())
    assert np.array_equal(out[0], out[1])


def test_backward_euler_pseudo_time_couette_order_p_plus_1():
    """The paper's steady runs: backward Euler with large steps to the steady
    state, then the repaired eq. exact at order p + 1 (Couette, Kn = 1)."""
    UW = 1e-3
    for p in (1, 2):
        errs = []
        for ny in (2, 4, 8):
            c = cases.couette(1, ny, p, U=UW, velset=("gh", 4), kn=1.0)
            pr = cases.oracle_problem(c)
            s = cases.solver(c, "fp64")
            s.set_equilibrium(1.0, 0.0, 0.0, 0.0, 0)
            st = s.implicit_step(_tight(0, 5.0, newton_rtol=1e-9, newton_atol=1e-12, gmres_rtol=1e-6,
                                        gmres_restart=100, gmres_max_iter=5000), 12)
            print("ny=%d p=%d: Newton %d GMRES %d" % (ny, p, st.newton_iters, st.gmres_iters))
            _, ux, _ = s.moments()
            errs.append(pr.l2_error(ux, lambda x, y: couette.exact_ux(y, 1.0, UW, -UW)) / (2 * UW))
        rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
        print("BE pseudo-time p=%d" % p, errs, rates)
        assert np.all(rates > p + 1 - 0.15), (p, errs, rates)


def test_implicit_errors():
    from paper_2012_13487_gb300 import fedbm as fb
    c = _couette_small()
    s = cases.solver(c, "bf16")
    s.set_equilibrium(1.0, 0.0, 0.0, 1e-3, 1)
    with pytest.raises(fb.FedbmError) as e:
        s.implicit_step(_tight(0, 0.1), 1)
    assert e.value.code == fb.FEDBM_EINVAL
    s = cases.solver(c, "fp64")
    s.set_equilibrium(1.0, 0.0, 0.0, 1e-2, 1)
    with pytest.raises(fb.FedbmError) as e:   # one Newton correction cannot reach 1e-15 relative
        s.implicit_step(_tight(0, 1.0, newton_rtol=1e-15, newton_atol=0.0, newton_max_iter=1, gmres_rtol=1e-2), 1)
    assert e.value.code == fb.FEDBM_ENOCONV
    with pytest.raises(fb.FedbmError) as e:
        s.implicit_step(fb.implicit_params(fb.IMPLICIT_CUSTOM, 0.1, A=[[0.5, 0.1], [0.2, 0.5]], b=[0.5, 0.5]), 1)
    assert e.value.code == fb.FEDBM_EINVAL


@pytest.mark.parametrize("form", ["unstructured", "split"])
def test_backward_euler_on_other_meshes_and_forms(form):
    """The implicit path runs R through whatever stage kernel the solver has:
    an unstructured mesh, or the velocity-split cluster form."""
    if form == "unstructured":
        c = cases.unstructured(cases.cavity(0, 0, 2, velset=("gh", 3), kn=1.0), 3, 2, seed=61)
        tile = {}
    else:
        c = cases.couette(1, 2, 2, velset=("nc", 8), kn=1.0)
        tile = {"vsplit": 2}
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=2e-2, seed=15)
    dt = 10 * pr.dt
    s = cases.solver(c, "fp64", **tile)
    if form == "split":
        assert s.info.velocity_split == 2
    s.set_state(f0)
    s.implicit_step(_tight(0, dt), 1)
    f_or, _ = implicit.sdirk_step(pr, f0, dt, "be")
    assert cases.rel_max_err(s.state(), f_or) < 1e-10


def test_backward_euler_steady_cavity_matches_oracle_steady_state():
    """The paper's cavity route (backward Euler to the steady state) on a small
    Kn = 2 cavity, against the oracle's own steady solver (pseudo-time Newton
    with a dense Jacobian taken once): the two steady states agree."""
    c = cases.cavity(2, 2, 2, velset=("gh", 3), kn=2.0, U=0.1)
    pr = cases.oracle_problem(c)
    fs, res = dg.steady_state(pr, pr.equilibrium_state())
    assert res < 1e-11
    s = cases.solver(c, "fp64")
    s.set_equilibrium(1.0, 0.0, 0.0, 0.0, 0)
    # near the steady state G_0 = dt |R| shrinks towards the FP64 rounding of
    # dt R (~1e-12 here), so each step stops at an absolute 1e-10 instead
    st = s.implicit_step(_tight(0, 50.0, newton_rtol=1e-9, newton_atol=1e-10, gmres_rtol=1e-8,
                                gmres_restart=120, gmres_max_iter=4000), 30)
    print("steady cavity: Newton %d GMRES %d" % (st.newton_iters, st.gmres_iters))
    f = s.state()
    assert np.abs(pr.rhs(f)).max() < 1e-9
    assert np.abs(f - fs).max() < 1e-8


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_block_jacobi_preconditioner(prec):
    """Right preconditioning by the element-and-velocity blocks of I - dt J
    gives the same step (to the solver tolerance) with far fewer GMRES
    iterations."""
    c = cases.couette(1, 8, 2, velset=("gh", 4), kn=1.0)
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=2e-2, seed=16)
    out, its = [], []
    tol = dict(newton_rtol=1e-10, newton_atol=1e-13) if prec == "fp64" else \
        dict(newton_rtol=1e-5, newton_atol=1e-6, gmres_rtol=1e-5)
    for pc in (0, 1):
        s = cases.solver(c, prec)
        s.set_state(f0)
        st = s.implicit_step(_tight(0, 40 * pr.dt, preconditioner=pc, **tol), 2)
        assert st.converged == 1
        out.append(s.state())
        its.append(st.gmres_iters)
    print(prec, "GMRES iterations without / with block Jacobi:", its)
    assert its[1] * 3 < its[0]
    f_or = implicit.march(pr, f0, 40 * pr.dt, 2, "be")
    bound = 1e-10 if prec == "fp64" else 2e-6
    for f in out:
        assert cases.rel_max_err(f, f_or) < bound
