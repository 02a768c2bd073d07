"""GPU test of fedbm_mass_noalloc, the allocation-free mass diagnostic.

Some callers cannot allocate device memory while they run (their memory
belongs to another allocator, or a real-time loop cannot pay for cudaMalloc),
so the library offers this variant whose scratch is a fixed device array.
This file is named so that pytest collects it last."""
import numpy as np
import pytest

import cases

pytestmark = pytest.mark.gpu


def test_mass_noalloc_matches_fedbm_mass_on_two_calls():
    import torch

    from paper_2012_13487_gb300 import fedbm as fb

    c = cases.cavity(6, 5, 3, velset=("gh", 4), kn=1.0)
    s = cases.solver(c, "fp64")
    s.set_equilibrium(1.0, 0.02, -0.01, 0.05, 11)
    s.step(3)
    want = s.mass()
    K, Np, Q = s.shape
    f = torch.empty((K, Np, Q), dtype=torch.float64, device="cuda")
    fb.fedbm_get_state(s.h, f, True)
    torch.cuda.synchronize()
    colsum = torch.tensor(fb.fedbm_ref_operators(3)["M"].sum(axis=0), dtype=torch.float64, device="cuda")
    jac = torch.full((K,), (1.0 / 6.0) * (1.0 / 5.0) / 4.0, dtype=torch.float64, device="cuda")
    total = torch.zeros(1, dtype=torch.float64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for scale in (1.0, 1.5):          # two calls in a row; the second sees a different state
        fb.fedbm_mass_noalloc(f * scale, jac, colsum, K, Np, Q, total, status, stream)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert float(total.item()) == pytest.approx(scale * want, rel=1e-13)
    # element Jacobians that differ from element to element: the per-element
    # factor of every node is taken from its own element
    rng = np.random.default_rng(7)
    jac_h = (0.5 + rng.random(K)) * (1.0 / 120.0)
    f_h = f.cpu().numpy()
    cs_h = colsum.cpu().numpy()
    want_nu = float(np.sum(jac_h[:, None] * cs_h[None, :] * f_h.sum(axis=-1)))
    jac_nu = torch.tensor(jac_h, dtype=torch.float64, device="cuda")
    for _ in range(2):
        fb.fedbm_mass_noalloc(f, jac_nu, colsum, K, Np, Q, total, status, stream)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert float(total.item()) == pytest.approx(want_nu, rel=1e-13)
    # a non-finite value is reported through the status word, then cleared again
    g = f.clone()
    g[2, 1, 3] = float("nan")
    fb.fedbm_mass_noalloc(g, jac, colsum, K, Np, Q, total, status, stream)
    torch.cuda.synchronize()
    assert int(status.item()) == 1
    fb.fedbm_mass_noalloc(f, jac, colsum, K, Np, Q, total, status, stream)
    torch.cuda.synchronize()
    assert int(status.item()) == 0 and float(total.item()) == pytest.approx(want, rel=1e-13)
    # beyond the fixed scratch capacity the call is refused before any launch
    with pytest.raises(fb.FedbmError) as e:
        fb.fedbm_mass_noalloc(f, jac, colsum, 2 ** 21, 2, Q, total, status, stream)
    assert e.value.code == fb.FEDBM_EINVAL
    s.close()
