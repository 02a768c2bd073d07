"""The CUDA path reproduces the paper's spatial order of accuracy (Sec. III.A):
Couette flow at Kn = 1 with D2Q16, marched to steady state on the GPU, against
the linearized closed form (eq. exact, repaired), converges at order p + 1."""
import numpy as np
import pytest

import cases
from oracle import couette

pytestmark = pytest.mark.gpu

UW = 1e-3


def steady_ux_error(ny, p, precision="fp64"):
    c = cases.couette(1, ny, p, U=UW, velset=("gh", 4), kn=1.0, cfl=0.5)
    pr = cases.oracle_problem(c)
    s = cases.solver(c, precision)
    s.set_equilibrium(1.0, 0.0, 0.0, 0.0, 0)
    dt = s.info.dt
    chunk = max(1, int(round(2.0 / dt)))          # two time units per check
    last = None
    for _ in range(40):                            # at most t = 80
        s.step(chunk)
        _, ux, _ = s.moments()
        if last is not None and np.abs(ux - last).max() < 1e-11 * UW / 1e-3:
            break
        last = ux
    err = pr.l2_error(ux, lambda x, y: couette.exact_ux(y, 1.0, UW, -UW)) / (2 * UW)
    return err


@pytest.mark.parametrize("p", [1, 2])
def test_couette_order_p_plus_1_on_gpu(p):
    errs = [steady_ux_error(ny, p) for ny in (2, 4, 8)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > p + 1 - 0.15), (errs, rates)
