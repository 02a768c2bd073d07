"""The CUDA path on unstructured triangulations (Sec. III.B runs the cavity
on unstructured meshes; a seeded jittered mesh with random diagonals, rotated
vertex lists and shuffled element order stands in for the paper's mesh file).
The stage kernels read every neighbour through the general face codes, so the
same kernels serve these meshes; each case is compared with the FP64 oracle
on the same mesh, element by element."""
import numpy as np
import pytest

from tests import cases

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def fp32_tol(pr, stages):
    return 4.0 * pr.Np * U32 * np.sqrt(stages) + U32


def _pair(c, nsteps, precision, amp=1e-2, seed=5, reduction="default", **tile):
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=amp, seed=seed)
    s = cases.solver(c, precision, reduction, **tile)
    s.set_state(f0)
    s.step(nsteps)
    return pr, s, f0, s.state(), pr.run(f0, nsteps)


@pytest.mark.parametrize("p", [1, 3, 5])
def test_unstructured_cavity_fp64(p):
    c = cases.unstructured(cases.cavity(0, 0, p, velset=("gh", 4), kn=8.0, eq_order=3), 6, 5, seed=31)
    pr, s, f0, f, f_or = _pair(c, 10, "fp64")
    assert s.info.K == 60
    assert cases.rel_max_err(f, f_or) < 1e-12
    m0 = pr.mass(f0)
    assert abs(s.mass() - m0) < 1e-13 * m0          # diffuse walls conserve mass


@pytest.mark.parametrize("vs,p", [(("nc", 16), 4), (("nc", 8), 2), (("gh", 4), 5)])
def test_unstructured_fp32_both_forms(vs, p):
    c = cases.unstructured(cases.cavity(0, 0, p, velset=vs, kn=1.0), 5, 5, seed=7)
    for tc in (-1, 1):
        if tc == 1 and vs[1] ** 2 not in (16, 256):
            continue
        pr, s, f0, f, f_or = _pair(c, 6, "fp32", tc=tc)
        assert s.info.tensor_cores == (1 if tc == 1 else 0)
        assert cases.rel_max_err(f, f_or) < fp32_tol(pr, 30)


def test_unstructured_periodic_couette_fp32():
    c = cases.unstructured(cases.couette(0, 0, 3, velset=("gh", 4), kn=1.0), 4, 6, seed=13)
    pr, s, f0, f, f_or = _pair(c, 8, "fp32")
    assert cases.rel_max_err(f, f_or) < fp32_tol(pr, 40)


@pytest.mark.parametrize("prec,u", [("bf16", 2.0 ** -8), ("fp16", 2.0 ** -11)])
def test_unstructured_deviation_forms(prec, u):
    c = cases.unstructured(cases.cavity(0, 0, 3, velset=("nc", 16), kn=8.0), 5, 4, seed=17)
    pr, s, f0, f, f1 = _pair(c, 2, prec, reduction="fp64")
    w = pr.w[None, None, :]
    md = np.abs(f1 / w - 1.0).max(axis=(1, 2))[:, None, None]
    assert (np.abs(f - f1) / (w * md)).max() < 12 * u


def test_batch_mixes_structured_and_unstructured_cases():
    from paper_2012_13487_gb300 import fedbm as fb
    cs = [cases.unstructured(cases.cavity(0, 0, 3, velset=("gh", 4), kn=2.0), 6, 4, seed=41),
          cases.cavity(4, 4, 3, velset=("gh", 4), kn=2.0),
          cases.unstructured(cases.couette(0, 0, 3, velset=("gh", 4), kn=0.5), 3, 5, seed=43)]
    b = cases.batch(cs, "fp32")
    prs = [cases.oracle_problem(c) for c in cs]
    f0s = [cases.initial_state(pr, amp=1e-2, seed=3 + j) for j, pr in enumerate(prs)]
    for j, f0 in enumerate(f0s):
        b.set_state(j, f0)
    b.step(4)
    assert b.info(0).ngroups == 1                    # one kernel group: same degree and velocity set
    for j, c in enumerate(cs):
        s = cases.solver(c, "fp32")
        s.set_state(f0s[j])
        s.step(4)
        got = b.state(j)
        assert np.array_equal(s.state(), got)
        assert cases.rel_max_err(got, prs[j].run(f0s[j], 4)) < fp32_tol(prs[j], 20)
