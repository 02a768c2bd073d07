"""GPU parity of the CUDA stage kernel (through the C ABI) against the FP64 oracle.

Tolerances:
* FP64 mode: max |f_gpu - f_oracle| / max |f_oracle| <= 1e-12 after the full
  run (the only differences are summation order and FMA contraction).
* FP32 mode: the state is rounded to FP32 (u = 2^-24) on every stage; the
  residual's dominant rounding is in the Dr/Ds contractions, whose terms are
  O(p^2 |f|) while the result is O(|grad f|).  One stage contributes at most
  about dt * |e| * |rx| * 2 Np * p^2 * u * max|f| ~ CFL * 2 Np * u * max|f|
  ~ Np * 6e-8 * max|f|; over S stages with random-walk accumulation the
  bound used is 4 * Np * u * sqrt(S) * max|f| (plus the u of the initial
  rounding).
* Deviation forms: reported L2 errors of rho and u against the oracle,
  bounded as stated per test.
"""
import numpy as np
import pytest

import cases

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _run_pair(c, nsteps, precision="fp32", amp=1e-3, seed=201213487, reduction="default", **tile):
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=amp, seed=seed)
    s = cases.solver(c, precision, reduction, **tile)
    s.set_state(f0)
    s.step(nsteps)
    f_gpu = s.state()
    f_or = pr.run(f0, nsteps)
    return pr, s, f0, f_gpu, f_or


def fp32_tol(pr, stages):
    return 4.0 * pr.Np * U32 * np.sqrt(stages) + U32


def test_couette_fp64_eq3_200_steps_parity():
    """Plain method in FP64: Couette Kn=1, GH D2Q16, third-order f^eq,
    8x8x2 mesh, p=2, diffuse walls at -+0.1, perturbation 1e-3, CFL 0.5,
    200 LSRK(5,4) steps."""
    c = cases.couette(8, 8, 2, U=0.1, velset=("gh", 4), eq_order=3, kn=1.0, cfl=0.5)
    pr, s, f0, f_gpu, f_or = _run_pair(c, 200, "fp64")
    assert s.info.dt == pytest.approx(pr.dt, rel=1e-15)
    err = cases.rel_max_err(f_gpu, f_or)
    assert err <= 1e-12, err
    rho, ux, uy = s.moments()
    orho, oux, ouy = pr.nodal_moments(f_or)
    assert np.abs(rho - orho).max() < 1e-12 and np.abs(ux - oux).max() < 1e-12
    assert s.mass() == pytest.approx(pr.mass(f_or), rel=1e-13)


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4, 5, 6])
def test_fp64_every_order_cavity(p):
    c = cases.cavity(3, 2, p, velset=("gh", 4), kn=2.0)
    pr, s, f0, f_gpu, f_or = _run_pair(c, 5, "fp64", amp=0.05)
    assert cases.rel_max_err(f_gpu, f_or) <= 1e-12


@pytest.mark.parametrize("c", [
    cases.cavity(5, 3, 4, velset=("gh", 4), kn=1.0),                 # ragged element tail
    cases.cavity(4, 3, 3, velset=("nc", 16), kn=8.0),                 # Q = 256
    cases.couette(3, 5, 5, velset=("gh", 4), eq_order=3, kn=0.5),
    cases.couette(2, 3, 2, velset=("gh", 3), kn=1.0),                 # D2Q9, Q padded 9 -> 16
    cases.cavity(2, 2, 3, velset=("nc", 32), kn=8.0),                 # Q = 1024
    dict(cases.cavity(3, 3, 2, velset=("gh", 4)), bc=("eq",) * 4),   # eq. UsedBC walls
    dict(cases.couette(3, 3, 3, velset=("gh", 4)), beta=0.5),         # central flux
    dict(nx=3, ny=3, p=2, bc=("periodic",) * 4, wall_u=((0, 0),) * 4, collision=False),
], ids=["gh16-p4-ragged", "nc256-p3", "gh16-p5-eq3", "d2q9-p2", "nc1024-p3", "usedbc", "central",
        "advection"])
def test_fp32_parity(c):
    n = 10
    pr, s, f0, f_gpu, f_or = _run_pair(c, n, "fp32", amp=0.05)
    err = cases.rel_max_err(f_gpu, f_or)
    assert err <= fp32_tol(pr, 5 * n), (err, fp32_tol(pr, 5 * n))


@pytest.mark.parametrize("epc,tpb,stages", [(1, 32, 1), (3, 64, 2), (8, 128, 1), (16, 256, 2), (5, 96, 2),
                                            (1, 32, 2)])
def test_fp32_tile_shapes_agree(epc, tpb, stages):
    c = cases.cavity(5, 4, 3, velset=("gh", 4), kn=1.0)
    pr, s, f0, f_gpu, f_or = _run_pair(c, 4, "fp32", amp=0.05, epc=epc, tpb=tpb, stages=stages)
    assert s.info.elems_per_cta == epc and s.info.threads_per_cta == tpb
    assert s.info.pipeline_stages == stages
    assert cases.rel_max_err(f_gpu, f_or) <= fp32_tol(pr, 20)


def test_pipelined_tiles_fp32_oracle():
    """Two tile buffers per CTA against the oracle."""
    c = cases.cavity(6, 5, 3, velset=("nc", 16), kn=8.0)
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=0.05)
    s = cases.solver(c, "fp32", stages=2, epc=1, tpb=128)
    assert s.info.pipeline_stages == 2
    s.set_state(f0)
    s.step(3)
    assert cases.rel_max_err(s.state(), pr.run(f0, 3)) <= fp32_tol(pr, 15)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_pipelined_persistent_tiles(prec):
    """Two tile buffers per CTA and fewer CTAs than tiles: each CTA loops over
    several tiles, loading the next one while it computes the current one;
    the result is bitwise that of the single-buffer schedule."""
    c = cases.cavity(32, 32, 3, velset=("nc", 16), kn=8.0)
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=0.05)
    ref = cases.solver(c, prec, stages=1, epc=1, tpb=256)
    s = cases.solver(c, prec, stages=2, epc=1, tpb=256)
    assert s.info.pipeline_stages == 2 and s.info.grid < s.info.K
    for x in (ref, s):
        x.set_state(f0)
        x.step(3)
    np.testing.assert_array_equal(s.state(), ref.state())


@pytest.mark.parametrize("red", ["fp64", "comp"])
def test_fp32_reduction_modes(red):
    c = cases.cavity(3, 3, 3, velset=("nc", 16), kn=1.0)
    pr, s, f0, f_gpu, f_or = _run_pair(c, 5, "fp32", amp=0.05, reduction=red)
    assert cases.rel_max_err(f_gpu, f_or) <= fp32_tol(pr, 25)


def test_set_equilibrium_matches_oracle_draw():
    c = cases.couette(4, 3, 3, velset=("gh", 4), eq_order=3)
    pr = cases.oracle_problem(c)
    s = cases.solver(c, "fp64")
    s.set_equilibrium(1.02, 0.03, -0.01, 1e-3, 201213487)
    want = cases.initial_state(pr, amp=1e-3, seed=201213487, rho0=1.02, ux0=0.03, uy0=-0.01)
    # same formula on both sides; only FMA contraction and operation order differ
    np.testing.assert_allclose(s.state(), want, rtol=4e-15, atol=0)


def test_single_stages_and_residual():
    c = cases.cavity(4, 3, 3, velset=("gh", 4), kn=1.0)
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=0.05)
    s = cases.solver(c, "fp64")
    s.set_state(f0)
    res = np.zeros_like(f0)
    f = f0
    for st in range(5):
        s.stage(st)
        f, res = pr.lsrk_stage(st, f, res)
        assert cases.rel_max_err(s.state(), f) < 1e-13
        assert np.abs(s.residual() - res).max() < 1e-13 * np.abs(f).max()


def test_mass_conserved_fp64_and_nonfinite_detected():
    c = cases.cavity(4, 4, 2, velset=("gh", 4), kn=1.0)
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=1e-3)
    s = cases.solver(c, "fp64")
    s.set_state(f0)
    m0 = s.mass()
    assert m0 == pytest.approx(pr.mass(f0), rel=1e-14)
    s.step(50)
    assert abs(s.mass() - m0) < 1e-13
    bad = f0.copy()
    bad[3, 2, 5] = np.nan
    s.set_state(bad)
    from paper_2012_13487_gb300 import fedbm as fb
    with pytest.raises(fb.FedbmError) as e:
        s.mass()
    assert e.value.code == fb.FEDBM_ENONFINITE


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_mass_diagnostic_fp64_of_the_stored_state(prec):
    """The mass diagnostic sums every stored value in FP64: for FP32 or 16-bit
    state it equals the FP64 mass of the decoded state to FP64 rounding."""
    c = cases.cavity(5, 4, 4, velset=("nc", 16), kn=1.0)
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=1e-2, seed=29)
    s = cases.solver(c, prec)
    s.set_state(f0)
    s.step(7)
    got = s.mass()
    want = pr.mass(s.state())
    assert abs(got - want) < 1e-14 * abs(want), (got, want)


# about twice the errors measured on the GB300 for this seeded case (L2 rho,
# L2 u/U after 20 steps): BF16 5.66e-6, 1.53e-4; FP16 5.00e-7, 5.95e-6;
# FP32 7.2e-8, 5.1e-7 (every moment-reduction mode within 0.5 % of these)
L2_BOUNDS_20_STEPS = {"bf16": (1.2e-5, 3.1e-4), "fp16": (1.0e-6, 1.2e-5), "fp32": (1.5e-7, 1.0e-6)}


@pytest.mark.parametrize("prec,red", [(p, r) for p in ("bf16", "fp16", "fp32") for r in ("default", "fp64", "comp")])
def test_deviation_forms_l2_error(prec, red):
    """Reduced-precision storage: L2 error of rho and u against the FP64
    oracle after 20 steps, relative to the lid speed (rho: absolute)."""
    c = cases.cavity(4, 4, 3, velset=("nc", 16), kn=8.0, U=0.1)
    pr, s, f0, f_gpu, f_or = _run_pair(c, 20, prec, amp=1e-3, reduction=red)
    rho, ux, uy = s.moments()
    orho, oux, ouy = pr.nodal_moments(f_or)
    e_rho = pr.l2_error(rho - orho, lambda x, y: 0 * x)
    e_u = np.hypot(pr.l2_error(ux - oux, lambda x, y: 0 * x), pr.l2_error(uy - ouy, lambda x, y: 0 * x)) / 0.1
    b_rho, b_u = L2_BOUNDS_20_STEPS[prec]
    assert e_rho < b_rho and e_u < b_u, (e_rho, e_u)


@pytest.mark.parametrize("tc", [1, -1])
def test_full_size_cavity_nc16_sampled_two_stages(tc):
    """Cavity Kn=1, 64x64x2, p=4, NC 16x16 (31.5M DOF) in the benchmark's
    launch configurations (the tensor-core form, and the FMA form with the
    autotuner's usual tile of one element and 128 threads): stages 0 and 1 on
    the GPU, compared on sampled elements with the oracle evaluated on just
    those elements."""
    c = cases.cavity(64, 64, 4, velset=("nc", 16), kn=1.0, U=0.1)
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=1e-2, seed=7)
    s = cases.solver(c, "fp32", tc=tc) if tc == 1 else cases.solver(c, "fp32", epc=1, tpb=128, stages=1)
    assert s.info.tensor_cores == (1 if tc == 1 else 0)
    s.set_state(f0)
    s.stage(0)
    f1_gpu = s.state()
    s.stage(1)
    f2_gpu = s.state()
    rng = np.random.default_rng(0)
    K = pr.K
    corners = [0, 1, 2 * 63, 2 * 63 + 1, K - 2, K - 1, K - 128, K - 127]
    sample = np.unique(np.concatenate([corners, rng.choice(K, 56, replace=False)]))
    ring = np.unique(np.concatenate([sample, pr.nbr_elem[sample][pr.nbr_elem[sample] >= 0]]))
    f1_ring, r1_ring = pr.lsrk_stage(0, f0, np.zeros((len(ring), pr.Np, pr.Q)), ring)
    f1 = f0.copy()
    f1[ring] = f1_ring
    r1 = np.zeros_like(f0)
    r1[ring] = r1_ring
    f2_s, _ = pr.lsrk_stage(1, f1, r1[sample], sample)
    scale = np.abs(f0).max()
    tol = fp32_tol(pr, 2) * scale
    assert np.abs(f1_gpu[sample] - f1[sample]).max() <= tol
    assert np.abs(f2_gpu[sample] - f2_s).max() <= tol


@pytest.mark.parametrize("vs,p,sqrt2", [(("nc", 33), 3, True), (("gh", 18), 2, False)])
def test_largest_velocity_sets_fp32(vs, p, sqrt2):
    """The paper's largest sets (NC 33x33 = D2Q1089 on the sqrt(2RT) grid,
    GH D2Q324) through the runtime-stride kernel: 1089 and 324 velocities pad to
    1096 and 328 (no compile-time stride)."""
    c = cases.cavity(2, 2, p, velset=vs, kn=2.0, nc_sqrt2=sqrt2)
    pr, s, f0, f_gpu, f_or = _run_pair(c, 2, "fp32", amp=1e-2)
    assert s.info.Q == vs[1] ** 2 and s.info.Q_padded % 8 == 0 and s.info.velocity_split == 1
    assert cases.rel_max_err(f_gpu, f_or) < fp32_tol(pr, 10)


@pytest.mark.parametrize("tc", [1, -1])
def test_full_size_cavity_nc16_bf16_sampled_two_stages(tc):
    """The BF16 deviation form of the same 31.5M-DOF cavity (the benchmark's
    BF16 form) in both kernel forms: stages 0 and 1, compared on sampled
    elements against the FP64 oracle within the 16-bit storage bound (12 u of
    w times the element's largest deviation, u = 2^-8)."""
    c = cases.cavity(64, 64, 4, velset=("nc", 16), kn=1.0, U=0.1)
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=1e-2, seed=8)
    s = cases.solver(c, "bf16", tc=tc)
    assert s.info.tensor_cores == (1 if tc == 1 else 0)
    s.set_state(f0)
    s.stage(0)
    s.stage(1)
    f2_gpu = s.state()
    rng = np.random.default_rng(1)
    K = pr.K
    sample = np.unique(np.concatenate([[0, 1, K - 2, K - 1], rng.choice(K, 28, replace=False)]))
    ring = np.unique(np.concatenate([sample, pr.nbr_elem[sample][pr.nbr_elem[sample] >= 0]]))
    f1_ring, r1_ring = pr.lsrk_stage(0, f0, np.zeros((len(ring), pr.Np, pr.Q)), ring)
    f1 = f0.copy()
    f1[ring] = f1_ring
    r1 = np.zeros_like(f0)
    r1[ring] = r1_ring
    f2_s, _ = pr.lsrk_stage(1, f1, r1[sample], sample)
    w = pr.w[None, None, :]
    md = np.abs(f2_s / w - 1.0).max(axis=(1, 2))[:, None, None]
    assert (np.abs(f2_gpu[sample] - f2_s) / (w * md)).max() < 12 * 2.0 ** -8


def test_full_size_couette_p5_gh16_sampled_two_stages():
    """Couette Kn=1, 256x256x2, p=5, GH D2Q16 (44M DOF, the convergence sweep's
    largest case) in its launch configuration: stages 0 and 1 on sampled
    elements, including both walls and the periodic seam."""
    c = cases.couette(256, 256, 5, velset=("gh", 4), kn=1.0, U=0.1)
    pr = cases.oracle_problem(c)
    f0 = cases.initial_state(pr, amp=1e-2, seed=9)
    s = cases.solver(c, "fp32")
    s.set_state(f0)
    s.stage(0)
    f1_gpu = s.state()
    s.stage(1)
    f2_gpu = s.state()
    rng = np.random.default_rng(2)
    K = pr.K
    edges = [0, 1, 2 * 255, 2 * 255 + 1, K - 2, K - 1, K - 512, K - 511]  # walls and the periodic seam
    sample = np.unique(np.concatenate([edges, rng.choice(K, 40, replace=False)]))
    ring = np.unique(np.concatenate([sample, pr.nbr_elem[sample][pr.nbr_elem[sample] >= 0]]))
    f1_ring, r1_ring = pr.lsrk_stage(0, f0, np.zeros((len(ring), pr.Np, pr.Q)), ring)
    f1 = f0.copy()
    f1[ring] = f1_ring
    r1 = np.zeros_like(f0)
    r1[ring] = r1_ring
    f2_s, _ = pr.lsrk_stage(1, f1, r1[sample], sample)
    tol = fp32_tol(pr, 2) * np.abs(f0).max()
    assert np.abs(f1_gpu[sample] - f1[sample]).max() <= tol
    assert np.abs(f2_gpu[sample] - f2_s).max() <= tol


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp64"])
def test_set_state_from_fp32_input(prec):
    """fedbm_set_state_f32 stores an FP32 state as fedbm_set_state stores the
    same values given in FP64 (bit for bit), from host and from device memory."""
    import torch

    from paper_2012_13487_gb300 import fedbm as fb
    c = cases.cavity(4, 3, 3, velset=("nc", 8), kn=1.0)
    pr = cases.oracle_problem(c)
    f32 = cases.initial_state(pr, amp=1e-2, seed=19).astype(np.float32)
    a = cases.solver(c, prec)
    a.set_state(f32.astype(np.float64))
    a.step(2)
    want = a.state()
    for on_device in (False, True):
        b = cases.solver(c, prec)
        src = torch.from_numpy(f32).cuda() if on_device else np.ascontiguousarray(f32)
        fb.fedbm_set_state_f32(b.h, src, on_device)
        torch.cuda.synchronize()
        b.step(2)
        assert np.array_equal(b.state(), want)
