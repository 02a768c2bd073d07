"""Tensor-core form of the stage kernel (tcgen05 TF32 MMAs with a hi/lo split
for the Dr, Ds and LIFT contractions) against the FP64 oracle and against the
FMA form, on the shapes it serves: FP32 state or BF16/FP16 deviation state,
128, 256 or 1024 padded velocities, degree <= 5, and 16 velocities (FP32, BF16)
with eight elements stacked into one 128-row MMA tile."""
import numpy as np
import pytest

from tests import cases

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def fp32_tol(pr, stages):
    return 4.0 * pr.Np * U32 * np.sqrt(stages) + U32


def _pair(c, nsteps, amp=1e-2, seed=17, reduction="default", **tile):
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=amp, seed=seed)
    s = cases.solver(c, "fp32", reduction, **tile)
    s.set_state(f0)
    s.step(nsteps)
    return pr, s, f0, s.state()


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_tc_cavity_nc16_matches_oracle_and_fma(p):
    c = cases.cavity(5, 4, p, velset=("nc", 16), kn=1.0)
    pr, s, f0, f_tc = _pair(c, 6, tc=1)
    assert s.info.tensor_cores == 1 and s.info.threads_per_cta == 128 and s.info.elems_per_cta == 1
    f_or = pr.run(f0, 6)
    assert cases.rel_max_err(f_tc, f_or) < fp32_tol(pr, 30)
    _, s2, _, f_fma = _pair(c, 6, tc=-1)
    assert s2.info.tensor_cores == 0
    assert cases.rel_max_err(f_tc, f_fma) < fp32_tol(pr, 30)


def test_tc_128_velocities_couette_eq3_usedbc_central():
    # NC 11x11 = 121 velocities padded to 128: one MMA tile, 128 threads
    c = cases.couette(6, 3, 3, velset=("nc", 11), eq_order=3, kn=0.5, beta=0.5)
    c["bc"] = ("eq", "periodic", "eq", "periodic")
    pr, s, f0, f_tc = _pair(c, 8, tc=1)
    assert s.info.tensor_cores == 1 and s.info.Q_padded == 128 and s.info.threads_per_cta == 128
    assert cases.rel_max_err(f_tc, pr.run(f0, 8)) < fp32_tol(pr, 40)


@pytest.mark.parametrize("p", [2, 4])
def test_tc_1024_velocities_cavity_kn8(p):
    # NC 32x32: eight 128-velocity passes per element
    c = cases.cavity(3, 3, p, velset=("nc", 32), kn=8.0)
    pr, s, f0, f_tc = _pair(c, 3, tc=1)
    assert s.info.tensor_cores == 1 and s.info.Q_padded == 1024
    assert cases.rel_max_err(f_tc, pr.run(f0, 3)) < fp32_tol(pr, 15)


def test_tc_default_selection_and_rejection():
    from paper_2012_13487_gb300 import fedbm as fb
    # the untuned default is the FMA form everywhere; tensor cores on request
    assert cases.solver(cases.cavity(3, 3, 4, velset=("nc", 16)), "fp32").info.tensor_cores == 0
    assert cases.solver(cases.cavity(3, 3, 4, velset=("nc", 16)), "fp32", tc=1).info.tensor_cores == 1
    assert cases.solver(cases.cavity(3, 3, 4, velset=("nc", 16)), "fp32", epc=2).info.tensor_cores == 0
    assert cases.solver(cases.cavity(3, 3, 4, velset=("gh", 5)), "fp32").info.tensor_cores == 0
    assert cases.solver(cases.cavity(3, 3, 4, velset=("nc", 16)), "bf16").info.tensor_cores == 0
    assert cases.solver(cases.cavity(3, 3, 4, velset=("nc", 16)), "bf16", tc=1).info.tensor_cores == 1
    assert cases.solver(cases.cavity(3, 3, 4, velset=("nc", 16)), "fp64").info.tensor_cores == 0
    assert cases.solver(cases.cavity(3, 3, 4, velset=("nc", 16)), "fp16").info.tensor_cores == 0
    assert cases.solver(cases.cavity(3, 3, 4, velset=("nc", 16)), "fp16", tc=1).info.tensor_cores == 1
    assert cases.solver(cases.cavity(3, 3, 5, velset=("nc", 16)), "fp32").info.tensor_cores == 0
    assert cases.solver(cases.cavity(3, 3, 5, velset=("nc", 16)), "fp32", tc=1).info.tensor_cores == 1
    assert cases.solver(cases.cavity(3, 3, 6, velset=("nc", 16)), "fp32").info.tensor_cores == 0
    with pytest.raises(fb.FedbmError) as e:   # 25 velocities padded to 32: no tensor-core form
        cases.solver(cases.cavity(3, 3, 4, velset=("gh", 5)), "fp32", tc=1)
    assert e.value.code == fb.FEDBM_EINVAL


@pytest.mark.parametrize("red", ["fp64", "comp"])
def test_tc_reductions(red):
    c = cases.cavity(4, 4, 3, velset=("nc", 16), kn=8.0)
    pr, s, f0, f = _pair(c, 4, seed=3, reduction=red, tc=1)
    assert s.info.tensor_cores == 1
    assert cases.rel_max_err(f, pr.run(f0, 4)) < fp32_tol(pr, 20)


def test_tc_collision_off():
    c = cases.couette(4, 4, 2, velset=("nc", 16), collision=False)
    pr, s, f0, f = _pair(c, 5, tc=1)
    assert cases.rel_max_err(f, pr.run(f0, 5)) < fp32_tol(pr, 25)


def test_tc_mass_conserved_long_run():
    c = cases.cavity(8, 8, 4, velset=("nc", 16), kn=1.0)
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=1e-3, seed=9)
    s = cases.solver(c, "fp32", tc=1)
    s.set_state(f0)
    m0 = s.mass()
    s.step(200)
    assert abs(s.mass() - m0) < 2e-5 * abs(m0)


def test_tc_wait_timeout_reported():
    from paper_2012_13487_gb300 import fedbm as fb
    c = cases.cavity(3, 2, 2, velset=("nc", 16))
    s = cases.solver(c, "fp32", tc=1, test_wait_timeout=1)
    assert s.info.tensor_cores == 1
    s.set_equilibrium(1.0, 0.0, 0.0, 1e-3, 5)
    s.stage(0)
    with pytest.raises(fb.FedbmError) as e:
        s.mass()
    assert e.value.code == fb.FEDBM_ETIMEOUT
    with pytest.raises(fb.FedbmError) as e:
        s.moments()
    assert e.value.code == fb.FEDBM_ETIMEOUT
    s.close()
    # every CTA released its tensor memory: the context still runs the
    # tensor-core form correctly
    pr, g, f0, f_tc = _pair(c, 3, tc=1)
    assert g.info.tensor_cores == 1
    assert cases.rel_max_err(f_tc, pr.run(f0, 3)) < fp32_tol(pr, 15)


def test_tc_batch_groups_toggle_bitwise_with_single_solvers():
    from paper_2012_13487_gb300 import fedbm as fb
    cs = [cases.cavity(4, 3, 4, velset=("nc", 16), kn=1.0), cases.couette(5, 2, 2, velset=("nc", 16), kn=2.0),
          cases.cavity(3, 3, 3, velset=("gh", 5))]
    # tensor cores requested for the first two cases (two groups), default for the third
    tcs = [1, 1, 0]
    b = fb.Batch([fb.case_desc(*cases.descriptors(c, "fp32", tc=t)) for c, t in zip(cs, tcs)])
    prs = [cases.oracle_problem(c) for c in cs]
    f0s = [cases.initial_state(pr, amp=1e-2, seed=21 + j) for j, pr in enumerate(prs)]
    for j, f0 in enumerate(f0s):
        b.set_state(j, f0)
    b.step(5)
    got = [b.state(j) for j in range(3)]
    infos = [b.info(j) for j in range(3)]
    assert [i.tensor_cores for i in infos] == [1, 1, 0]
    for j, c in enumerate(cs):
        s = cases.solver(c, "fp32", tc=tcs[j])
        s.set_state(f0s[j])
        s.step(5)
        assert np.array_equal(s.state(), got[j])
    # switch the first group to the FMA form and back
    g = infos[0].group
    fb.fedbm_batch_set_tensor_cores(b.h, g, 0)
    assert b.info(0).tensor_cores == 0
    fb.fedbm_batch_set_tensor_cores(b.h, g, 1)
    assert b.info(0).tensor_cores == 1


@pytest.mark.parametrize("prec,u", [("bf16", 2.0 ** -8), ("fp16", 2.0 ** -11)])
@pytest.mark.parametrize("p,vs", [(4, ("nc", 16)), (3, ("nc", 32))])
def test_tc_deviation_forms(prec, u, p, vs):
    """16-bit deviation state on the tensor-core form: after 2 steps every value
    is within the storage bound of the 16-bit parity tests of the oracle
    (12 encodings' worth of u relative to w times the element's largest
    deviation), and the tensor-core and FMA forms agree to that bound too."""
    c = cases.cavity(4, 3, p, velset=vs, kn=8.0)
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=1e-2, seed=41)
    out = {}
    for tc in (1, -1):
        s = cases.solver(c, prec, "fp64", tc=tc)
        assert s.info.tensor_cores == (1 if tc == 1 else 0)
        s.set_state(f0)
        s.step(2)
        out[tc] = s.state()
        s.mass()
    f1 = pr.run(f0, 2)
    w = pr.w[None, None, :]
    md = np.abs(f1 / w - 1.0).max(axis=(1, 2))[:, None, None]
    for tc in (1, -1):
        assert (np.abs(out[tc] - f1) / (w * md)).max() < 12 * u
    assert (np.abs(out[1] - out[-1]) / (w * md)).max() < 12 * u


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("nx,ny", [(4, 4), (3, 3)])   # 32 elements, and 18 (a ragged last tile of 2)
def test_tc_stacked_gh16_fp32(p, nx, ny):
    c = cases.cavity(nx, ny, p, velset=("gh", 4), kn=1.0, eq_order=3)
    pr, s, f0, f_tc = _pair(c, 6, tc=1)
    assert s.info.tensor_cores == 1 and s.info.Q_padded == 16 and s.info.elems_per_cta == 8
    assert cases.rel_max_err(f_tc, pr.run(f0, 6)) < fp32_tol(pr, 30)
    _, _, _, f_fma = _pair(c, 6, tc=-1)
    assert cases.rel_max_err(f_tc, f_fma) < fp32_tol(pr, 30)


def test_tc_stacked_gh16_couette_bf16():
    c = cases.couette(5, 3, 3, velset=("gh", 4), kn=0.5)
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=1e-2, seed=43)
    s = cases.solver(c, "bf16", tc=1)
    assert s.info.tensor_cores == 1 and s.info.elems_per_cta == 8
    s.set_state(f0)
    s.step(2)
    f1 = pr.run(f0, 2)
    w = pr.w[None, None, :]
    md = np.abs(f1 / w - 1.0).max(axis=(1, 2))[:, None, None]
    assert (np.abs(s.state() - f1) / (w * md)).max() < 12 * 2.0 ** -8
