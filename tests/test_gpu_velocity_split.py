"""Velocity-split form of the stage kernel (a thread-block cluster of CTAs
per element tile, each CTA one slice of the velocities; the node moments and
the eq. FullBC wall numerators are summed across the cluster through
distributed shared memory).  It opens the paper's largest velocity set, NC
33 x 33 = D2Q1089 on the sqrt(2RT) grid (Sec. III.B), at degrees 5 and 6,
where one CTA cannot hold an element's velocities; every case is compared with
the FP64 oracle element by element, and the split and unsplit forms with
each other where both exist."""
import numpy as np
import pytest

from tests import cases

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def fp32_tol(pr, stages):
    return 4.0 * pr.Np * U32 * np.sqrt(stages) + U32


def _run(c, nsteps, precision, amp=1e-2, seed=23, reduction="default", **tile):
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=amp, seed=seed)
    s = cases.solver(c, precision, reduction, **tile)
    s.set_state(f0)
    s.step(nsteps)
    return pr, s, f0, s.state()


@pytest.mark.parametrize("ncl", [2, 4, 8])
def test_forced_split_fp64_matches_oracle_and_unsplit(ncl):
    c = cases.cavity(3, 2, 3, velset=("nc", 16), kn=2.0, eq_order=3)
    pr, s, f0, f = _run(c, 4, "fp64", vsplit=ncl)
    assert s.info.velocity_split == ncl
    f_or = pr.run(f0, 4)
    assert cases.rel_max_err(f, f_or) < 1e-12
    _, s1, _, f1 = _run(c, 4, "fp64", vsplit=1)
    assert s1.info.velocity_split == 1
    assert cases.rel_max_err(f, f1) < 1e-13


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_forced_split_reduced_precision(prec):
    c = cases.couette(4, 3, 4, velset=("nc", 16), kn=1.0)
    pr, s, f0, f = _run(c, 3, prec, vsplit=4)
    assert s.info.velocity_split == 4
    f_or = pr.run(f0, 3)
    if prec == "fp32":
        assert cases.rel_max_err(f, f_or) < fp32_tol(pr, 15)
    else:
        w = pr.w[None, None, :]
        md = np.abs(f_or / w - 1.0).max(axis=(1, 2))[:, None, None]
        assert (np.abs(f - f_or) / (w * md)).max() < 12 * 2.0 ** -8


@pytest.mark.parametrize("p", [5, 6])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_d2q1089_at_high_degree(p, prec):
    """D2Q1089 pads to 1120 velocities; at degrees 5 and 6 the automatic rule
    takes the velocity-split form."""
    c = cases.cavity(2, 2, p, velset=("nc", 33), kn=2.0, nc_sqrt2=True)
    pr, s, f0, f = _run(c, 1, prec, amp=1e-2)
    assert s.info.Q == 1089 and s.info.Q_padded == 1120
    # one CTA holds a BF16 element of degree 5 (181 KB), not one of degree 6 or in FP32
    assert s.info.velocity_split >= 2 or (prec == "bf16" and p == 5)
    f_or = pr.run(f0, 1)
    if prec == "fp32":
        assert cases.rel_max_err(f, f_or) < fp32_tol(pr, 5)
    else:
        w = pr.w[None, None, :]
        md = np.abs(f_or / w - 1.0).max(axis=(1, 2))[:, None, None]
        assert (np.abs(f - f_or) / (w * md)).max() < 12 * 2.0 ** -8
    s.mass()


def test_d2q1089_fp64_split_and_mass():
    c = cases.cavity(2, 1, 5, velset=("nc", 33), kn=8.0, nc_sqrt2=True)
    pr, s, f0, f = _run(c, 2, "fp64", amp=1e-2)
    assert s.info.velocity_split >= 2
    assert cases.rel_max_err(f, pr.run(f0, 2)) < 1e-12
    assert abs(s.mass() - pr.mass(f0)) < 1e-13


def test_split_wait_timeout_reported_and_context_usable():
    from paper_2012_13487_gb300 import fedbm as fb
    c = cases.cavity(2, 2, 2, velset=("nc", 16), kn=1.0)
    s = cases.solver(c, "fp32", vsplit=2, test_wait_timeout=1)
    assert s.info.velocity_split == 2
    s.set_equilibrium(1.0, 0.0, 0.0, 1e-3, 5)
    s.stage(0)
    with pytest.raises(fb.FedbmError) as e:
        s.mass()
    assert e.value.code == fb.FEDBM_ETIMEOUT
    s.close()
    pr, g, f0, f = _run(c, 2, "fp32", vsplit=2)
    assert cases.rel_max_err(f, pr.run(f0, 2)) < fp32_tol(pr, 10)


def test_split_rejections():
    from paper_2012_13487_gb300 import fedbm as fb
    c = cases.cavity(2, 2, 2, velset=("gh", 5), kn=1.0)     # 25 -> 32 velocities: no 8-multiple slices of 8 CTAs
    with pytest.raises(fb.FedbmError):
        cases.solver(c, "fp32", vsplit=8)
    with pytest.raises(fb.FedbmError):
        cases.solver(cases.cavity(2, 2, 2, velset=("nc", 16)), "fp16", vsplit=2)


def test_split_on_an_unstructured_mesh():
    c = cases.unstructured(cases.cavity(0, 0, 3, velset=("nc", 16), kn=2.0), 4, 3, seed=51)
    pr, s, f0, f = _run(c, 3, "fp64", vsplit=4)
    assert s.info.velocity_split == 4
    assert cases.rel_max_err(f, pr.run(f0, 3)) < 1e-12
