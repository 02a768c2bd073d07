"""The warp-specialised stage kernel (pipeline_stages = 3) against the FP64 oracle.

The form computes the same stage as the FMA kernel (Sec. II.B.1 residual,
LSRK(5,4) update) with a producer warp keeping a three-stage ring of element
tiles ahead of eight consumer warps.  It exists for FP32 and BF16 state with
256 padded velocities (the NC 16x16 sets, GH D2Q256) at degree <= 5.
Tolerances are those of the FMA kernel's tests: the FP32 bound
4 Np u sqrt(S) + u (u = 2^-24) over S stages, and for BF16 12 u of w times the
element's largest deviation (u = 2^-8).
"""
import time

import numpy as np
import pytest

import cases

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def fp32_tol(pr, stages):
    return 4.0 * pr.Np * U32 * np.sqrt(stages) + U32


def _ws_solver(c, prec="fp32", **kw):
    s = cases.solver(c, prec, stages=3, **kw)
    i = s.info
    assert i.pipeline_stages == 3 and i.threads_per_cta == 288 and i.elems_per_cta == 1
    assert i.tensor_cores == 0 and i.velocity_split == 1
    return s


def _bf16_norm_err(pr, f, f_ref):
    w = pr.w[None, None, :]
    md = np.abs(f_ref / w - 1.0).max(axis=(1, 2))[:, None, None]
    return float((np.abs(f - f_ref) / (w * md)).max())


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4, 5])
def test_ws_fp32_every_degree_cavity(p):
    n = 3 if p < 5 else 2
    c = cases.cavity(n, n, p, velset=("nc", 16), kn=1.0)
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=0.05, seed=31 + p)
    s = _ws_solver(c)
    s.set_state(f0)
    s.step(4)
    err = cases.rel_max_err(s.state(), pr.run(f0, 4))
    assert err <= fp32_tol(pr, 20), err


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4, 5])
def test_ws_bf16_every_degree_cavity(p):
    """The BF16 form's volume contractions on the tensor cores (q against
    [Dr; Ds] in three BF16 pieces) at every degree, against the oracle within
    the 16-bit storage bound and against the FMA kernel's BF16 form to a few
    storage units."""
    n = 3 if p < 5 else 2
    c = cases.cavity(n, n, p, velset=("nc", 16), kn=1.0)
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=0.05, seed=61 + p)
    out = []
    for s in (_ws_solver(c, "bf16"), cases.solver(c, "bf16", stages=1, epc=1, tpb=128)):
        s.set_state(f0)
        s.step(2)
        out.append(s.state())
        s.close()
    e_or, d = _bf16_norm_err(pr, out[0], pr.run(f0, 2)), _bf16_norm_err(pr, out[0], out[1])
    print("p=%d bf16 ws: vs oracle %.3e, vs fma %.3e (units of w md)" % (p, e_or, d))
    assert e_or < 12 * 2.0 ** -8
    assert d <= 4 * 2.0 ** -8


@pytest.mark.parametrize("c", [
    cases.couette(3, 4, 3, velset=("nc", 16), kn=0.5),                    # periodic seam + walls
    cases.couette(3, 3, 2, velset=("gh", 16), eq_order=3, kn=1.0),        # GH D2Q256, third order
    dict(cases.cavity(3, 3, 2, velset=("nc", 16)), bc=("eq",) * 4),      # eq. UsedBC walls
    dict(cases.couette(3, 3, 3, velset=("nc", 16)), beta=0.5),            # central flux
    dict(nx=3, ny=3, p=2, velset=("nc", 16), bc=("periodic",) * 4, wall_u=((0, 0),) * 4, collision=False),
    cases.unstructured(cases.cavity(0, 0, 3, velset=("nc", 16), kn=2.0), 4, 3),
], ids=["couette", "gh256-eq3", "usedbc", "central", "advection", "unstructured"])
def test_ws_fp32_cases(c):
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=0.05, seed=41)
    s = _ws_solver(c)
    s.set_state(f0)
    s.step(5)
    err = cases.rel_max_err(s.state(), pr.run(f0, 5))
    assert err <= fp32_tol(pr, 25), err


@pytest.mark.parametrize("red", ["default", "fp64", "comp"])
def test_ws_reduction_modes(red):
    c = cases.cavity(3, 3, 3, velset=("nc", 16), kn=1.0)
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=0.05, seed=43)
    s = _ws_solver(c, reduction=red)
    s.set_state(f0)
    s.step(5)
    assert cases.rel_max_err(s.state(), pr.run(f0, 5)) <= fp32_tol(pr, 25)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_ws_ring_wraps_and_matches_fma_kernel(prec):
    """Fewer CTAs than elements: each CTA walks many elements through its ring
    (the stages are refilled many times over).  The result agrees with the FMA
    kernel and with the oracle: FP32 to a few units of rounding (the same
    arithmetic); BF16 to a few storage units, since this form takes the volume
    contractions on q (tensor cores), the FMA kernel on the decoded f, and an
    encode that rounds the other way in one stage carries into the next."""
    c = cases.cavity(40, 40, 3, velset=("nc", 16), kn=8.0)
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=0.05, seed=44)
    ws = _ws_solver(c, prec)
    assert ws.info.grid < ws.info.K // 4
    fma = cases.solver(c, prec, stages=1, epc=1, tpb=128)
    out = []
    for s in (ws, fma):
        s.set_state(f0)
        s.step(2)
        out.append(s.state())
    f_or = pr.run(f0, 2)
    if prec == "fp32":
        scale = np.abs(f_or).max()
        print("ws vs fma max |df| / max|f| = %.3e" % (np.abs(out[0] - out[1]).max() / scale))
        assert np.abs(out[0] - out[1]).max() <= 8 * U32 * scale
        assert cases.rel_max_err(out[0], f_or) <= fp32_tol(pr, 10)
    else:
        d = _bf16_norm_err(pr, out[0], out[1])
        print("ws vs fma bf16: max |df| / (w md) = %.3e" % d)
        assert d <= 4 * 2.0 ** -8
        assert _bf16_norm_err(pr, out[0], f_or) < 12 * 2.0 ** -8


def test_ws_bf16_stochastic_rounding_matches_fma_kernel():
    """The stochastic BF16 encode draws the same counter-based numbers in both
    forms (value index, step, stage), so the states agree to a few storage
    units (the contractions round differently) and stay within the storage
    bound of the oracle."""
    c = cases.cavity(6, 6, 3, velset=("nc", 16), kn=8.0)
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=1e-3, seed=45)
    out = []
    for s in (_ws_solver(c, "bf16", rounding=1), cases.solver(c, "bf16", stages=1, epc=1, tpb=128, rounding=1)):
        s.set_state(f0)
        s.step(3)
        out.append(s.state())
        s.close()
    assert _bf16_norm_err(pr, out[0], out[1]) <= 4 * 2.0 ** -8
    assert _bf16_norm_err(pr, out[0], pr.run(f0, 3)) < 12 * 2.0 ** -8


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_ws_full_size_cavity_nc16_sampled_two_stages(prec):
    """Cavity Kn=1, 64x64x2, p=4, NC 16x16 (31.5M DOF) in this form: stages 0
    and 1 on the GPU, compared on sampled elements (corners, walls and random
    ones) with the oracle evaluated on just those elements."""
    c = cases.cavity(64, 64, 4, velset=("nc", 16), kn=1.0, U=0.1)
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=1e-2, seed=46)
    s = _ws_solver(c, prec)
    s.set_state(f0)
    s.stage(0)
    f1_gpu = s.state()
    s.stage(1)
    f2_gpu = s.state()
    s.close()
    rng = np.random.default_rng(3)
    K = pr.K
    corners = [0, 1, 2 * 63, 2 * 63 + 1, K - 2, K - 1, K - 128, K - 127]
    sample = np.unique(np.concatenate([corners, rng.choice(K, 40, replace=False)]))
    ring = np.unique(np.concatenate([sample, pr.nbr_elem[sample][pr.nbr_elem[sample] >= 0]]))
    f1_ring, r1_ring = pr.lsrk_stage(0, f0, np.zeros((len(ring), pr.Np, pr.Q)), ring)
    f1 = f0.copy()
    f1[ring] = f1_ring
    r1 = np.zeros_like(f0)
    r1[ring] = r1_ring
    f2_s, _ = pr.lsrk_stage(1, f1, r1[sample], sample)
    if prec == "fp32":
        tol = fp32_tol(pr, 2) * np.abs(f0).max()
        assert np.abs(f1_gpu[sample] - f1[sample]).max() <= tol
        assert np.abs(f2_gpu[sample] - f2_s).max() <= tol
    else:
        assert _bf16_norm_err(pr, f2_gpu[sample], f2_s) < 12 * 2.0 ** -8


def test_ws_implicit_step_matches_fma_form():
    """The implicit solver's residual evaluations run on whichever stage form
    the solver holds; one backward-Euler step agrees with the FMA form's to the
    Newton tolerance."""
    from paper_2012_13487_gb300 import fedbm as fb
    c = cases.couette(2, 4, 2, velset=("nc", 16), kn=1.0)
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=1e-2, seed=47)
    out = []
    for s in (_ws_solver(c), cases.solver(c, "fp32", stages=1)):
        s.set_state(f0)
        st = s.implicit_step(fb.implicit_params(fb.IMPLICIT_BE, 10 * pr.dt, newton_rtol=1e-5, newton_atol=1e-6,
                                                gmres_rtol=1e-5), 1)
        assert st.converged == 1
        out.append(s.state())
        s.close()
    assert cases.rel_max_err(out[0], out[1]) < 2e-6


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_ws_wait_timeout_reported_and_context_usable(prec):
    """The test hook (16 expected bytes that never arrive) makes the consumers'
    bounded wait on the first ring stage run out; they record the timeout and
    leave (the BF16 form releasing its tensor memory first), the producer's
    bounded wait on the stage release runs out too, and the host reads
    FEDBM_ETIMEOUT.  The context stays usable."""
    from paper_2012_13487_gb300 import fedbm as fb
    c = cases.cavity(4, 4, 2, velset=("nc", 16), kn=1.0)
    s = _ws_solver(c, prec, test_wait_timeout=1)
    s.set_equilibrium(1.0, 0.0, 0.0, 1e-3, 5)
    t0 = time.time()
    s.stage(0)
    with pytest.raises(fb.FedbmError) as e:
        s.mass()
    assert e.value.code == fb.FEDBM_ETIMEOUT
    assert time.time() - t0 < 60.0
    s.close()
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=1e-3, seed=5)
    g = _ws_solver(c, prec)   # for BF16: allocates tensor memory again
    g.set_state(f0)
    g.step(1)
    if prec == "fp32":
        assert cases.rel_max_err(g.state(), pr.run(f0, 1)) <= fp32_tol(pr, 5)
    else:
        assert _bf16_norm_err(pr, g.state(), pr.run(f0, 1)) < 12 * 2.0 ** -8


def test_ws_unsupported_forms_rejected():
    from paper_2012_13487_gb300 import fedbm as fb
    nc = cases.cavity(2, 2, 2, velset=("nc", 16))
    for prec in ("fp64", "fp16"):
        with pytest.raises(fb.FedbmError) as e:
            cases.solver(nc, prec, stages=3)
        assert e.value.code == fb.FEDBM_EINVAL
    with pytest.raises(fb.FedbmError) as e:
        cases.solver(cases.cavity(2, 2, 2, velset=("gh", 4)), "fp32", stages=3)   # 16 velocities
    assert e.value.code == fb.FEDBM_EINVAL
    with pytest.raises(fb.FedbmError) as e:
        cases.solver(cases.cavity(1, 1, 6, velset=("nc", 16)), "fp32", stages=3)  # degree 6
    assert e.value.code == fb.FEDBM_EINVAL


def test_ws_in_a_batch_by_set_tiles():
    """A batch group re-tiled to this form (and a group of another velocity
    count that cannot take it, which keeps its tile) steps like the oracle."""
    from paper_2012_13487_gb300 import fedbm as fb
    cs = [cases.cavity(4, 3, 3, velset=("nc", 16), kn=1.0), cases.cavity(5, 5, 3, velset=("nc", 16), kn=4.0),
          cases.couette(3, 2, 2, velset=("gh", 4), kn=1.0)]
    b = cases.batch(cs, "fp32")
    g_nc, g_gh = b.info(0).group, b.info(2).group
    assert b.info(1).group == g_nc and g_gh != g_nc
    fb.fedbm_batch_set_tiles(b.h, g_nc, 0, 0, 3)
    before = (b.info(2).elems_per_cta, b.info(2).threads_per_cta, b.info(2).pipeline_stages)
    with pytest.raises(fb.FedbmError):
        fb.fedbm_batch_set_tiles(b.h, g_gh, 0, 0, 3)
    assert (b.info(2).elems_per_cta, b.info(2).threads_per_cta, b.info(2).pipeline_stages) == before
    assert b.info(0).pipeline_stages == 3 and b.info(1).pipeline_stages == 3
    prs = [cases.oracle_problem(c) for c in cs]
    f0s = [cases.initial_state(pr, amp=0.05, seed=50 + j) for j, pr in enumerate(prs)]
    for j, f0 in enumerate(f0s):
        b.set_state(j, f0)
    b.step(3)
    for j, (pr, f0) in enumerate(zip(prs, f0s)):
        assert cases.rel_max_err(b.state(j), pr.run(f0, 3)) <= fp32_tol(pr, 15)
    b.close()


def test_autotune_times_the_ws_candidate(tmp_path):
    """The autotuner times this form among its candidates for 256 velocities
    and keeps whichever runs fastest; the kept configuration steps correctly."""
    c = cases.cavity(16, 16, 4, velset=("nc", 16), kn=1.0)
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=0.05, seed=52)
    s = cases.solver(c, "fp32")
    path = tmp_path / "tune.json"
    s.autotune(str(path), 3)
    print("autotuned:", path.read_text().strip())
    s.set_state(f0)
    s.step(2)
    assert cases.rel_max_err(s.state(), pr.run(f0, 2)) <= fp32_tol(pr, 10)
