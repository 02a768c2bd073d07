"""The measurement arithmetic of bench.py, on the CPU.

The metric is DOF-stage updates per second; the roofline divides the
algorithmic bytes of one stage launch (state read and write, residual read
and write, the first of the five LSRK(5,4) stages reading no residual) by the
average launch time; recorded DRAM traffic is taken from a committed ncu
summary only when that summary was captured on the current kernel sources,
for the same kernel form and state precision."""
import glob
import os

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("prec,want", [("fp64", 152), ("fp32", 76), ("bf16", 56), ("fp16", 56)])
def test_algorithmic_bytes_per_dof_step(prec, want):
    s, r = bench.STATE_BYTES[prec], bench.RES_BYTES[prec]
    # stage 1: f read + f write + res write; stages 2-5: f and res read and written
    assert bench.algorithmic_bytes_per_dof_step(prec) == (2 * s + r) + 4 * (2 * s + 2 * r) == want


def test_default_workload_dimensions():
    w = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]
    assert bench.dims(w) == (2 * 64 * 64, 15, 256)
    K, Np, Q = bench.dims(w)
    assert K * Np * Q == 31_457_280


def test_roofline_of_is_bytes_over_launch_time():
    dof, ms = 31_457_280, 0.52
    r = bench.roofline_of(dof, "fp32", ms, "stage_kernel_ws")
    alg = dof * 76
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(alg / 5)
    # five launches per step: bytes per launch over the time per launch
    assert r["achieved"] == pytest.approx((alg / 5) / (ms / 5 * 1e-3) / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    peak, kind = bench.hbm_peak()
    assert r["peak"] == peak and r["peak_source"] == kind
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert kind == "measured"
    else:
        assert (peak, kind) == (bench.FALLBACK_HBM_GBS, "fallback")


def test_spread_of_repeats():
    sp = bench.spread([10.0, 12.0, 11.0], 10)
    assert sp["n"] == 3 and sp["ms_per_step_median"] == pytest.approx(1.1)
    assert sp["ms_per_step_min"] == pytest.approx(1.0) and sp["ms_per_step_max"] == pytest.approx(1.2)
    assert sp["spread_pct"] == pytest.approx(100 * 0.2 / 1.1)


def test_recorded_traffic_only_for_the_current_sources_and_form():
    sha = bench.stage_kernel_sha()
    seen_current = False
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "stage_kernel_*.md"))):
        name = os.path.basename(path)[len("stage_kernel_"):-3]
        txt = open(path).read()
        fields = dict(line.split(":", 1) for line in txt.splitlines()
                      if line.split(":", 1)[0] in ("kernel_source_sha256_16", "kernel", "precision",
                                                   "dram_bytes_per_launch"))
        kern, prec = fields["kernel"].strip(), fields["precision"].strip()
        got = bench.recorded_traffic(name, kern, prec)
        if fields["kernel_source_sha256_16"].strip() == sha:
            seen_current = True
            assert got == float(fields["dram_bytes_per_launch"])
            # another form or precision does not borrow the figure
            assert bench.recorded_traffic(name, kern + "_other", prec) is None
            assert bench.recorded_traffic(name, kern, "fp64") is None
        else:
            assert got is None
    if not seen_current:
        pytest.skip("no ncu summary was captured on the current stage-kernel sources")


def test_kernel_source_hash_ignores_comments_and_blank_space(tmp_path, monkeypatch):
    src = os.path.join(ROOT, "paper_2012_13487_gb300", "csrc")
    names = ("stage_impl.cuh", "stage_tc.cuh", "stage_cluster.cuh", "stage_ws.cuh", "device_common.cuh")
    dst = tmp_path / "paper_2012_13487_gb300" / "csrc"
    dst.mkdir(parents=True)
    for n in names:
        (dst / n).write_text(open(os.path.join(src, n)).read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.stage_kernel_sha()
    # comments added, line breaks doubled, indentation widened: the same code
    (dst / "stage_ws.cuh").write_text("// a comment\n\n" + (dst / "stage_ws.cuh").read_text()
                                      .replace("\n", "  // note\n\n").replace("\n  ", "\n    "))
    assert bench.stage_kernel_sha() == h0
    (dst / "stage_ws.cuh").write_text((dst / "stage_ws.cuh").read_text() + "\nint x;\n")
    assert bench.stage_kernel_sha() != h0


