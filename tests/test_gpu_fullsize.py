"""Full-size checks of the benchmark configurations that the other parity
tests only cover on reduced meshes: the 256-case batch (about 1.6G DOF),
the Kn = 8 BF16 cavity (128x128x2, p = 3, NC 32x32, 335M DOF) and the
GH D2Q16 cavity (64x64x2, p = 4, 1.97M DOF)."""
import numpy as np
import pytest

import bench
from oracle import dg
from tests import cases

pytestmark = pytest.mark.gpu


def test_full_batch256_sampled_cases_bitwise_as_single_solvers():
    """One step of the whole seeded 256-case batch; sampled cases (both kinds,
    both velocity sets, several degrees) equal single solvers bit for bit."""
    w = bench.WORKLOADS["batch256_couette_cavity_fp32"]
    cs = bench.batch_case_list(w)
    b = bench.make_batch(cs, 0)
    for i in range(len(cs)):
        b.set_equilibrium(i, 1.0, 0.0, 0.0, 1e-3, 201213487 + i)
    b.step(1)
    picks = sorted({0, 1, 63, 127, 128, 129, 200, 255})
    for i in picks:
        s = bench.make_solver(cs[i], 0)
        s.set_equilibrium(1.0, 0.0, 0.0, 1e-3, 201213487 + i)
        s.step(1)
        assert np.array_equal(s.state(), b.state(i)), (i, cs[i])
        s.close()
    b.close()


def test_full_size_cavity_kn8_bf16_stage0_sampled():
    """The 335M-DOF BF16 cavity in its default launch configuration: the
    device-generated initial state (the same SplitMix64 perturbation as the
    oracle's) and one stage, compared on sampled elements with the oracle
    within the 16-bit storage bound."""
    import torch

    c = cases.cavity(128, 128, 3, velset=("nc", 32), kn=8.0, U=0.1)
    pr = cases.oracle_problem(c)
    amp, seed = 1e-2, 77
    s = cases.solver(c, "bf16", "fp64")
    s.set_equilibrium(1.0, 0.0, 0.0, amp, seed)
    s.stage(0)
    K, Np, Q = s.shape
    f_dev = torch.empty((K, Np, Q), dtype=torch.float64, device="cuda")
    from paper_2012_13487_gb300 import fedbm as fb
    fb.fedbm_get_state(s.h, f_dev, True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    sample = np.unique(np.concatenate([[0, 1, 2 * 127, K - 2, K - 1], rng.choice(K, 19, replace=False)]))
    f1_gpu = f_dev[torch.as_tensor(sample, device="cuda")].cpu().numpy()
    del f_dev
    f0 = cases.initial_state(pr, amp=amp, seed=seed)
    f1_s, _ = pr.lsrk_stage(0, f0, np.zeros((len(sample), Np, Q)), sample)
    del f0
    w = pr.w[None, None, :]
    md = np.abs(f1_s / w - 1.0).max(axis=(1, 2))[:, None, None]
    assert (np.abs(f1_gpu - f1_s) / (w * md)).max() < 12 * 2.0 ** -8



@pytest.mark.parametrize("tc", [1, -1], ids=["tensor-cores", "fma"])
def test_full_size_cavity_gh16_three_steps(tc):
    """Cavity Kn=1, 64x64x2, p=4, GH D2Q16 (1.97M DOF): three whole LSRK(5,4)
    steps in both kernel forms, compared with the oracle on every value."""
    c = cases.cavity(64, 64, 4, velset=("gh", 4), kn=1.0, U=0.1)
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=1e-2, seed=12)
    s = cases.solver(c, "fp32", tc=tc)
    s.set_state(f0)
    s.step(3)
    err = cases.rel_max_err(s.state(), pr.run(f0, 3))
    tol = 4.0 * pr.Np * 2.0 ** -24 * np.sqrt(15) + 2.0 ** -24
    assert err <= tol, (err, tol)
    s.close()


def test_full_batch256_sampled_cases_against_the_oracle():
    """The seeded 256-case batch itself against the FP64 oracle: after one
    LSRK step of the whole batch from each case's seeded perturbed rest state,
    sampled cases (both kinds, both velocity sets, several degrees) are compared
    with the oracle's step on sampled elements, within the FP32 rounding bound
    of the parity tests."""
    from paper_2012_13487_gb300 import inputs
    w = bench.WORKLOADS["batch256_couette_cavity_fp32"]
    cs = bench.batch_case_list(w)
    b = bench.make_batch(cs, 0)
    for i in range(len(cs)):
        b.set_equilibrium(i, 1.0, 0.0, 0.0, 1e-3, 201213487 + i)
    picks = [0, 37, 127, 128, 190, 255]
    got = {}
    b.step(1)
    for i in picks:
        got[i] = b.state(i)
    b.close()
    rng = np.random.default_rng(4)
    for i in picks:
        c = cs[i]
        kind, n = c["vel"]
        bc = ("diffuse",) * 4 if c["kind"] == "cavity" else ("diffuse", "periodic", "diffuse", "periodic")
        wall = ((0, 0), (0, 0), (c["speed"], 0), (0, 0)) if c["kind"] == "cavity" else \
            ((-c["speed"], 0), (0, 0), (c["speed"], 0), (0, 0))
        pr = dg.Problem(c["nx"], c["ny"], c["p"], velset=(kind, n), kn=c["kn"], bc=bc, wall_u=wall)
        f0 = pr.equilibrium_state(amp=1e-3, u=inputs.perturbation(201213487 + i, pr.K, pr.Np, pr.Q))
        f1 = pr.run(f0, 1)
        elems = np.sort(rng.choice(pr.K, min(pr.K, 64), replace=False))
        err = np.abs(got[i][elems] - f1[elems]).max() / np.abs(f1).max()
        tol = 4.0 * pr.Np * 2.0 ** -24 * np.sqrt(5) + 2.0 ** -24
        assert err < tol, (i, c, err, tol)
