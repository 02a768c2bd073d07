"""GPU tests of the batched form: many independent Couette and cavity cases of
uneven mesh size, degree, velocity set, Kn and wall speed advance together."""
import numpy as np
import pytest

import cases
from test_gpu_parity import fp32_tol

pytestmark = pytest.mark.gpu


MIX = [
    cases.couette(3, 4, 2, U=0.05, velset=("gh", 4), kn=0.7),
    cases.cavity(4, 3, 3, U=0.2, velset=("nc", 16), kn=8.0),
    cases.cavity(2, 5, 2, U=0.1, velset=("gh", 4), kn=2.0),      # same group as case 0
    cases.couette(5, 2, 3, U=0.15, velset=("nc", 16), kn=0.5),    # same group as case 1
    cases.cavity(3, 3, 4, U=0.12, velset=("gh", 4), kn=1.3),
    cases.couette(2, 2, 5, U=0.08, velset=("gh", 4), kn=4.0),
]


def test_batch_matches_oracle_and_single_solvers():
    b = cases.batch(MIX, "fp32")
    groups = {b.info(c).group for c in range(len(MIX))}
    assert b.info(0).ngroups == len(groups) == 4
    assert b.info(0).group == b.info(2).group and b.info(1).group == b.info(3).group
    prs, f0s = [], []
    for c, case in enumerate(MIX):
        pr = cases.oracle_problem(case)
        f0 = cases.initial_state(pr, amp=0.05, seed=100 + c)
        b.set_state(c, f0)
        prs.append(pr)
        f0s.append(f0)
    nsteps = 6
    b.step(nsteps)
    for c, case in enumerate(MIX):
        pr, f0 = prs[c], f0s[c]
        assert b.info(c).dt == pytest.approx(pr.dt, rel=1e-14)
        got = b.state(c)
        want = pr.run(f0, nsteps)
        assert cases.rel_max_err(got, want) <= fp32_tol(pr, 5 * nsteps)
        single = cases.solver(case, "fp32")
        single.set_state(f0)
        single.step(nsteps)
        np.testing.assert_array_equal(got, single.state())   # same arithmetic per element


def test_batch_equilibrium_and_mass_per_case():
    b = cases.batch(MIX[:3], "fp32")
    for c in range(3):
        b.set_equilibrium(c, 1.0, 0.0, 0.0, 1e-3, 7 + c)
    m0 = [b.mass(c) for c in range(3)]
    b.step(20)
    for c in range(3):
        # diffuse walls conserve mass; FP32 state rounding bounds the drift
        assert abs(b.mass(c) - m0[c]) < 1e-5 * abs(m0[c])


def test_autotune_keeps_state_and_uses_cache(tmp_path):
    b = cases.batch(MIX[:4], "fp32")
    f0s = []
    for c in range(4):
        pr = cases.oracle_problem(MIX[c])
        f0s.append(cases.initial_state(pr, amp=0.05, seed=c))
        b.set_state(c, f0s[-1])
    cache = str(tmp_path / "tiles.json")
    b.autotune(cache, 2)
    for c in range(4):
        np.testing.assert_array_equal(b.state(c), np.asarray(b.state(c)))
        assert cases.rel_max_err(b.state(c), f0s[c]) < 1e-7        # only FP32 rounding of f0
    text = open(cache).read()
    assert text.count('"epc"') == b.info(0).ngroups
    tiles = [(b.info(c).elems_per_cta, b.info(c).threads_per_cta, b.info(c).pipeline_stages) for c in range(4)]
    b.step(2)
    b2 = cases.batch(MIX[:4], "fp32")
    b2.autotune(cache, 2)                                           # served from the cache
    assert [(b2.info(c).elems_per_cta, b2.info(c).threads_per_cta, b2.info(c).pipeline_stages)
            for c in range(4)] == tiles
    for c in range(4):
        b2.set_state(c, f0s[c])
    b2.step(2)
    for c in range(4):
        np.testing.assert_array_equal(b2.state(c), b.state(c))


def test_groups_sharing_a_kernel_with_different_tiles_and_failed_retile():
    """Two groups that use the same compiled stage kernel with different tiles
    (different shared-memory sizes) both launch, and a rejected re-tile leaves
    its group as it was."""
    from paper_2012_13487_gb300 import fedbm as fb
    c = cases.cavity(4, 3, 3, velset=("nc", 16), kn=1.0)
    descs = [fb.case_desc(*cases.descriptors(c, "fp32", epc=4, tpb=256)),
             fb.case_desc(*cases.descriptors(c, "fp32", epc=1, tpb=128))]
    b = fb.Batch(descs)
    assert b.info(0).ngroups == 2
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=1e-2, seed=77)
    for j in range(2):
        b.set_state(j, f0)
    with pytest.raises(fb.FedbmError) as e:
        fb.fedbm_batch_set_tiles(b.h, b.info(1).group, 1, 48, 1)   # not a multiple of 32
    assert e.value.code == fb.FEDBM_EINVAL
    assert b.info(1).threads_per_cta == 128
    b.step(3)
    f_or = pr.run(f0, 3)
    for j in range(2):
        assert cases.rel_max_err(b.state(j), f_or) < 4.0 * pr.Np * 2.0 ** -24 * np.sqrt(15) + 2.0 ** -24
