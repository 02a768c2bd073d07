"""The seeded input recipes (draws only, no arithmetic of the method).

The 256-case batch stands in for many independent Couette (Sec. III.A) and
cavity (Sec. III.B) runs of uneven size: the first half Couette, the rest
cavity; Kn log-uniform in [0.5, 8]; wall or lid speed uniform in
[0.05, 0.2]; N x N x 2 triangles with N in 16..64; degree 2..5; GH D2Q16 or
NC 16 x 16 with probability 1/2 each.  The per-value perturbation is a
function of the canonical index only, so it does not depend on any layout."""
import numpy as np

from paper_2012_13487_gb300 import inputs


def test_batch_recipe_ranges_and_split():
    cs = inputs.batch_cases()
    assert len(cs) == 256
    assert [c["kind"] for c in cs] == ["couette"] * 128 + ["cavity"] * 128
    kn = np.array([c["kn"] for c in cs])
    assert kn.min() >= 0.5 and kn.max() <= 8.0
    # log-uniform: log Kn is spread over the whole interval, about evenly
    lk = (np.log(kn) - np.log(0.5)) / (np.log(8.0) - np.log(0.5))
    assert np.histogram(lk, bins=4, range=(0, 1))[0].min() > 40
    assert all(0.05 <= c["speed"] <= 0.2 for c in cs)
    assert {c["p"] for c in cs} == {2, 3, 4, 5}
    assert min(c["N"] for c in cs) >= 16 and max(c["N"] for c in cs) <= 64
    assert {c["vel"] for c in cs} == {("gh", 4), ("nc", 16)}
    assert 100 < sum(c["vel"] == ("gh", 4) for c in cs) < 156


def test_batch_recipe_is_deterministic_and_seeded():
    assert inputs.batch_cases() == inputs.batch_cases()
    assert inputs.batch_cases(seed=1) != inputs.batch_cases()


def test_batch_total_size():
    # K = 2 N^2 elements, Np = (p + 1)(p + 2) / 2 nodes, 16 or 256 velocities:
    # about 1.6e9 DOF, the 13 GB of state and residual the batch workload moves
    dof = sum(2 * c["N"] ** 2 * (c["p"] + 1) * (c["p"] + 2) // 2 * (16 if c["vel"][0] == "gh" else 256)
              for c in inputs.batch_cases())
    assert dof == 1_605_736_320


def test_perturbation_depends_on_the_canonical_index_only():
    K, Np, Q = 7, 6, 16
    u = inputs.perturbation(42, K, Np, Q)
    assert u.shape == (K, Np, Q) and u.min() >= -1.0 and u.max() < 1.0
    flat = inputs.uniform_pm1(42, K * Np * Q)
    np.testing.assert_array_equal(u.ravel(), flat)
    # a later block of the same sequence starts where its canonical index says
    np.testing.assert_array_equal(inputs.uniform_pm1(42, 50, start=100), flat[100:150])
