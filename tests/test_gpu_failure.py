"""Failure detection and checkpoint/resume on the GPU.

The failure is made without faulting the GPU: a test hook makes every stage
kernel expect 16 bytes more than its tile copies bring, so the kernel's bounded
wait on the tile barrier runs out, the kernel records the timeout in the
solver's status word and returns.  The host reads the status through
fedbm_mass (FEDBM_ETIMEOUT), and the CUDA context stays usable: a second solver
in the same process then matches the oracle.

Checkpoint/resume: the state copied out after n steps and copied into a new
solver continues bit for bit as if the run had not stopped (stage 0 of the
low-storage scheme does not read the residual register, so a step boundary
needs no more than the state).
"""
import time

import numpy as np
import pytest

from tests import cases

pytestmark = pytest.mark.gpu


def _couette():
    return cases.couette(8, 2, 3, velset=("gh", 4), eq_order=3, kn=0.5)


def test_stage_wait_timeout_reported_and_context_usable():
    from paper_2012_13487_gb300 import fedbm as fb
    c = _couette()
    s = cases.solver(c, "fp32", epc=2, tpb=128, stages=1, test_wait_timeout=1)
    s.set_equilibrium(1.0, 0.0, 0.0, 1e-3, 5)
    t0 = time.time()
    s.stage(0)
    with pytest.raises(fb.FedbmError) as e:
        s.mass()
    assert e.value.code == fb.FEDBM_ETIMEOUT
    assert time.time() - t0 < 60.0
    # the synchronous host read-outs report it too, and it stays until a new state is loaded
    with pytest.raises(fb.FedbmError) as e:
        s.moments()
    assert e.value.code == fb.FEDBM_ETIMEOUT
    with pytest.raises(fb.FedbmError) as e:
        s.state()
    assert e.value.code == fb.FEDBM_ETIMEOUT
    with pytest.raises(fb.FedbmError) as e:
        s.mass()
    assert e.value.code == fb.FEDBM_ETIMEOUT
    s.set_equilibrium(1.0, 0.0, 0.0, 1e-3, 5)
    s.mass()
    s.moments()
    s.close()

    # the context still works: an ordinary solver matches the oracle
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=1e-3, seed=5)
    g = cases.solver(c, "fp64")
    g.set_state(f0)
    g.step(3)
    f_or = pr.run(f0, 3)
    assert cases.rel_max_err(g.state(), f_or) < 1e-12
    g.mass()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_checkpoint_resume_bitwise(prec):
    c = cases.cavity(6, 6, 2, velset=("nc", 8), kn=1.0)
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=1e-2, seed=11)
    a = cases.solver(c, prec)
    a.set_state(f0)
    a.step(30)
    ref = a.state()

    b = cases.solver(c, prec)
    b.set_state(f0)
    b.step(12)
    ckpt = b.state()
    b.close()
    r = cases.solver(c, prec)
    r.set_state(ckpt)
    r.step(18)
    assert np.array_equal(r.state(), ref)
