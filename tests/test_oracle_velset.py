"""Pins of the oracle's velocity sets (Sec. II.A.3, Table 1, Sec. III.B)."""
import os

import numpy as np
import pytest

from oracle import velset

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_table1_d1q4_d1q5_closed_forms():
    # Table 1: D1Q4 nodes +-sqrt(3 -+ sqrt6), weights (3 +- sqrt6)/12
    x, w = velset.gauss_hermite_1d(4)
    s6 = np.sqrt(6.0)
    np.testing.assert_allclose(np.sort(np.abs(x))[::2], [np.sqrt(3 - s6), np.sqrt(3 + s6)], rtol=1e-14)
    np.testing.assert_allclose(w[np.argsort(np.abs(x))][::2], [(3 + s6) / 12, (3 - s6) / 12], rtol=1e-14)
    # D1Q5: 0 (8/15), +-sqrt(5 -+ sqrt10) ((7 +- 2 sqrt10)/60)
    x, w = velset.gauss_hermite_1d(5)
    s10 = np.sqrt(10.0)
    order = np.argsort(np.abs(x))
    np.testing.assert_allclose(np.abs(x[order])[[0, 1, 3]], [0.0, np.sqrt(5 - s10), np.sqrt(5 + s10)], atol=1e-14)
    np.testing.assert_allclose(w[order][[0, 1, 3]], [8 / 15, (7 + 2 * s10) / 60, (7 - 2 * s10) / 60], rtol=1e-13)


def test_table1_d1q6_printed_values():
    # The printed D1Q6 values agree with the exact rule to about 12 digits
    # (the table's last printed digits are off by ~1e-12 relative), so the
    # printed numbers pin the rule to 1.5e-12; the exact nodes are pinned
    # separately by the roots of He_6(x) = x^6 - 15 x^4 + 45 x^2 - 15.
    rows = np.array(_load("table1_d1q6.txt"), dtype=np.float64)
    x, w = velset.gauss_hermite_1d(6)
    pos = x > 0
    np.testing.assert_allclose(np.sort(x[pos]), rows[:, 0], rtol=1.5e-12)
    np.testing.assert_allclose(w[pos][np.argsort(x[pos])], rows[:, 1], rtol=1.5e-12)
    he6_roots = np.sort(np.real(np.roots([1, 0, -15, 0, 45, 0, -15])))
    np.testing.assert_allclose(np.sort(x), he6_roots, rtol=1e-14)


@pytest.mark.parametrize("n", [3, 4, 5, 6, 8, 12, 18])
def test_gh_exact_to_degree_2n_minus_1(n):
    x, w = velset.gauss_hermite_1d(n)
    for k in range(2 * n):
        gauss_moment = 0.0 if k % 2 else float(np.prod(np.arange(k - 1, 0, -2))) if k else 1.0
        scale = np.sum(w * np.abs(x) ** k)      # size of the terms that cancel
        assert abs(np.sum(w * x ** k) - gauss_moment) <= 1e-13 * scale
    # one degree higher is no longer exact (the rule has degree exactly 2n-1)
    k = 2 * n
    assert abs(np.sum(w * x ** k) - float(np.prod(np.arange(k - 1, 0, -2)))) > 1e-6


def test_d2q9_matches_printed_set():
    rows = np.array(_load("d2q9.txt"), dtype=np.float64)
    ex, ey, w = velset.velocity_set("gh", 3)
    got = sorted(zip(np.round(ex / np.sqrt(3), 12), np.round(ey / np.sqrt(3), 12), np.round(w * 36, 12)))
    want = sorted(zip(rows[:, 0], rows[:, 1], rows[:, 2]))
    np.testing.assert_allclose(np.array(got), np.array(want), atol=1e-12)


def test_gh_d2q324_weight_underflow():
    row = [r for r in _load("weight_underflow.txt") if r[0] == "gh_d2q324"][0]
    _, _, w = velset.velocity_set("gh", int(row[1]))
    assert len(w) == 324
    assert int(np.sum(w < 2.2e-16)) == int(row[2])
    assert int(np.floor(np.log10(w.min()))) == int(row[3])


def test_nc_d2q1089_weight_underflow_sqrt2rt_grid():
    row = [r for r in _load("weight_underflow.txt") if r[0] == "nc_d2q1089"][0]
    _, _, w = velset.velocity_set("nc", int(row[1]), 4.0, np.sqrt(2.0))
    assert len(w) == 1089
    assert np.all(w > 0)
    assert int(np.sum(w < 2.2e-16)) == int(row[2])
    # on a grid in units of sqrt(RT) no weight underflows
    _, _, w1 = velset.velocity_set("nc", 33, 4.0, 1.0)
    assert int(np.sum(w1 < 2.2e-16)) == 0


@pytest.mark.parametrize("n,scale", [(16, 1.0), (32, 1.0), (33, np.sqrt(2.0)), (9, 1.0)])
def test_nc_even_moments_corrected(n, scale):
    x, w = velset.newton_cotes_1d(n, 4.0, scale)
    np.testing.assert_allclose(x, -x[::-1], atol=1e-15)
    assert np.all(w > 0)
    for k, m in ((0, 1.0), (2, 1.0), (4, 3.0)):
        assert abs(np.sum(w * x ** k) - m) < 1e-13
    for k in (1, 3, 5):
        assert abs(np.sum(w * x ** k)) < 1e-13


def test_tensor_index_convention():
    x, w = velset.gauss_hermite_1d(4)
    ex, ey, w2 = velset.tensor_2d(x, w)
    for ix in range(4):
        for iy in range(4):
            i = ix * 4 + iy
            assert ex[i] == x[ix] and ey[i] == x[iy] and w2[i] == w[ix] * w[iy]
