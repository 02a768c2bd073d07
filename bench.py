#!/usr/bin/env python
"""Throughput benchmark of the fused DG-FEM discrete-velocity BGK stage.

One "step" is one full LSRK(5,4) time step (five fused stage kernels) of the
whole mesh.  The metric is DOF-stage updates per second:
K * Np * Q * 5 * steps / time, a DOF being one (element, node, velocity) value.

Default workload: lid-driven cavity at Kn = 1 on a 64x64x2 triangle mesh,
p = 4 (15 nodes), 16x16 Newton-Cotes velocities on [-4, 4] sqrt(RT), lid
speed 0.1 sqrt(RT), diffuse walls, FP32, rest-equilibrium start (31.5M DOF;
the two state buffers and the residual, 378 MB, are larger than L2, so no L2
flush is needed between steps).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the FP64 CPU oracle on host cores

Under torchrun each rank runs an independent replica of the workload (the
solver needs no communication); the value is the sum over ranks of the
DOF-stage updates divided by the slowest rank's time.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "cavity_kn1_64x64x2_p4_nc16x16_fp32": dict(
        kind="cavity", nx=64, ny=64, p=4, vel=("nc", 16), kn=1.0, speed=0.1, precision="fp32",
        desc="lid-driven cavity Kn=1, 64x64x2 triangles, p=4, NC 16x16 on [-4,4]sqrt(RT), lid 0.1, FP32"),
    "cavity_kn1_64x64x2_p4_nc16x16_bf16": dict(
        kind="cavity", nx=64, ny=64, p=4, vel=("nc", 16), kn=1.0, speed=0.1, precision="bf16",
        desc="lid-driven cavity Kn=1, 64x64x2 triangles, p=4, NC 16x16 on [-4,4]sqrt(RT), lid 0.1, "
             "BF16 deviation state"),
    "cavity_kn1_64x64x2_p5_nc16x16_fp32": dict(
        kind="cavity", nx=64, ny=64, p=5, vel=("nc", 16), kn=1.0, speed=0.1, precision="fp32",
        desc="lid-driven cavity Kn=1, 64x64x2 triangles, p=5, NC 16x16 on [-4,4]sqrt(RT), lid 0.1, FP32"),
    "cavity_kn1_64x64x2_p4_gh16_fp32": dict(
        kind="cavity", nx=64, ny=64, p=4, vel=("gh", 4), kn=1.0, speed=0.1, precision="fp32",
        desc="lid-driven cavity Kn=1, 64x64x2 triangles, p=4, GH D2Q16, lid 0.1, FP32"),
    "couette_kn1_256x256x2_p5_gh16_fp32": dict(
        kind="couette", nx=256, ny=256, p=5, vel=("gh", 4), kn=1.0, speed=0.1, precision="fp32",
        desc="Couette Kn=1, 256x256x2 triangles, p=5, GH D2Q16, walls -+0.1, FP32"),
    "couette_kn1_256x256x2_p5_gh16_bf16": dict(
        kind="couette", nx=256, ny=256, p=5, vel=("gh", 4), kn=1.0, speed=0.1, precision="bf16",
        desc="Couette Kn=1, 256x256x2 triangles, p=5, GH D2Q16, walls -+0.1, BF16 deviation state"),
    "cavity_kn8_128x128x2_p3_nc32x32_bf16": dict(
        kind="cavity", nx=128, ny=128, p=3, vel=("nc", 32), kn=8.0, speed=0.1, precision="bf16",
        desc="lid-driven cavity Kn=8, 128x128x2 triangles, p=3, NC 32x32, BF16 deviation state, FP64 moments",
        reduction="fp64"),
}
WORKLOADS["cavity_kn2_64x64x2_p4_nc16x16_fp32"] = dict(
    kind="cavity", nx=64, ny=64, p=4, vel=("nc", 16), kn=2.0, speed=0.1, precision="fp32",
    desc="lid-driven cavity Kn=2, 64x64x2 triangles, p=4, NC 16x16 on [-4,4]sqrt(RT), lid 0.1, FP32")
WORKLOADS["cavity_kn1_unstructured_8192_p4_nc16x16_fp32"] = dict(
    kind="cavity", nx=64, ny=64, p=4, vel=("nc", 16), kn=1.0, speed=0.1, precision="fp32",
    unstructured=True, mesh_seed=201213487,
    desc="lid-driven cavity Kn=1, unstructured 8192-triangle mesh of the unit square (jittered 64x64 vertex "
         "grid, random diagonals), p=4, NC 16x16, lid 0.1, FP32")
WORKLOADS["cavity_kn8_32x32x2_p5_nc33x33_sqrt2_fp32"] = dict(
    kind="cavity", nx=32, ny=32, p=5, vel=("nc", 33), nc_sqrt2=1, kn=8.0, speed=0.1, precision="fp32",
    desc="lid-driven cavity Kn=8, 32x32x2 triangles, p=5, NC 33x33 = D2Q1089 on the sqrt(2RT) grid "
         "(velocity-split cluster kernel), lid 0.1, FP32")
WORKLOADS["batch256_couette_cavity_fp32"] = dict(
    kind="batch", seed=201213487, n=256, precision="fp32",
    desc="256 seeded independent cases (128 Couette, 128 cavity; Kn log-uniform in [0.5, 8], wall/lid "
         "speed in [0.05, 0.2], N x N x 2 triangles with N in 16..64, p in 2..5, GH D2Q16 or NC 16x16), FP32")
DEFAULT_WORKLOAD = "cavity_kn1_64x64x2_p4_nc16x16_fp32"
PREC = {"fp64": 0, "fp32": 1, "bf16": 2, "fp16": 3}
RED = {"default": 0, "fp64": 1, "comp": 2}
# algorithmic bytes per DOF for one stage: f read + res read + res write + f write
STATE_BYTES = {"fp64": 8, "fp32": 4, "bf16": 2, "fp16": 2}
RES_BYTES = {"fp64": 8, "fp32": 4, "bf16": 4, "fp16": 4}
FALLBACK_HBM_GBS = 6800.0


def algorithmic_bytes_per_dof_step(prec):
    """Five stages; the first has A = 0 and does not read the residual."""
    s, r = STATE_BYTES[prec], RES_BYTES[prec]
    return (2 * s + r) + 4 * (2 * s + 2 * r)


def batch_case_list(w):
    from paper_2012_13487_gb300 import inputs
    out = []
    for c in inputs.batch_cases(w["seed"], w["n"]):
        out.append(dict(kind=c["kind"], nx=c["N"], ny=c["N"], p=c["p"], vel=c["vel"], kn=c["kn"],
                        speed=c["speed"], precision=w["precision"]))
    return out


def dims(w):
    p = w["p"]
    Np = (p + 1) * (p + 2) // 2
    Q = w["vel"][1] ** 2
    K = 2 * w["nx"] * w["ny"]
    return K, Np, Q


def stage_kernel_sha():
    """Hash of the stage-kernel sources with comments and blank space removed,
    so that only code changes void a recorded ncu traffic figure."""
    h = hashlib.sha256()
    for n in ("stage_impl.cuh", "stage_tc.cuh", "stage_cluster.cuh", "stage_ws.cuh", "device_common.cuh"):
        with open(os.path.join(ROOT, "paper_2012_13487_gb300", "csrc", n)) as fh:
            code = re.sub(r"//[^\n]*", "", fh.read())
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(name, kernel, precision=None):
    """DRAM bytes per stage launch from the committed ncu summary, if it was
    taken for the current kernel source, the kernel form and the state
    precision this run times; else None."""
    path = os.path.join(ROOT, "profiles", "stage_kernel_%s.md" % name)
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m1 = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    m2 = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    m3 = re.search(r"^kernel:\s*(\S+)", txt, re.M)
    if not m1 or not m2 or m1.group(1) != stage_kernel_sha():
        return None
    if m3 and m3.group(1) != kernel:
        return None
    m4 = re.search(r"^precision:\s*(\S+)", txt, re.M)
    if precision and m4 and m4.group(1) != precision:
        return None
    return float(m2.group(1))


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        for key in ("hbm_gbs", "hbm_GBs", "hbm_copy_gbs"):
            if key in d:
                return float(d[key]), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_median": statistics.median(float(r[3]) for r in rows
                                                    if r[3].replace(".", "").isdigit()) if rows else None}


def make_descriptors(w, epc=0, tpb=0, stages=0, tc=0):
    from paper_2012_13487_gb300 import fedbm as fb
    if w["kind"] == "cavity":
        bc = (fb.BC_WALL_DIFFUSE,) * 4
        wall = ((0, 0), (0, 0), (w["speed"], 0), (0, 0))
    else:
        bc = (fb.BC_WALL_DIFFUSE, fb.BC_PERIODIC, fb.BC_WALL_DIFFUSE, fb.BC_PERIODIC)
        wall = ((-w["speed"], 0), (0, 0), (w["speed"], 0), (0, 0))
    if w.get("unstructured"):
        from paper_2012_13487_gb300 import inputs
        vert, tri = inputs.unstructured_square(w["nx"], w["ny"], w["mesh_seed"], shuffle=False)
        m = fb.unstructured_mesh_desc(vert, tri, w["p"], bc=bc, wall_u=wall)
    else:
        m = fb.mesh_desc(w["nx"], w["ny"], w["p"], bc=bc, wall_u=wall)
    kind, n = w["vel"]
    v = fb.velset_desc(fb.VELSET_GH if kind == "gh" else fb.VELSET_NC, n, eq_order=w.get("eq_order", 2),
                       nc_sqrt2=w.get("nc_sqrt2", 0))
    prm = fb.params(kn=w["kn"], precision=PREC[w["precision"]], reduction=RED[w.get("reduction", "default")],
                    cfl=0.5, elems_per_cta=epc, threads_per_cta=tpb, pipeline_stages=stages, tensor_cores=tc,
                    rounding=w.get("rounding", 0), velocity_split=w.get("velocity_split", 0))
    return m, v, prm


def make_solver(w, stream_handle, epc=0, tpb=0, stages=0, tc=0):
    from paper_2012_13487_gb300 import fedbm as fb
    return fb.Solver(*make_descriptors(w, epc, tpb, stages, tc), stream_handle)


def make_batch(cases, stream_handle):
    from paper_2012_13487_gb300 import fedbm as fb
    return fb.Batch([fb.case_desc(*make_descriptors(c)) for c in cases], stream_handle)


def time_steps(step, stream, steps, warmup):
    """Event time (ms) of `steps` calls of step(1) on `stream` after `warmup` calls."""
    import torch
    step(warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def measure_batch(w, stream, steps, warmup, loop_steps, tune):
    """Batched form and the case-by-case loop of single solvers on the same cases."""
    import torch
    cases = batch_case_list(w)
    dof = sum(2 * c["nx"] * c["ny"] * ((c["p"] + 1) * (c["p"] + 2) // 2) * c["vel"][1] ** 2 for c in cases)
    b = make_batch(cases, stream.cuda_stream)
    for i in range(len(cases)):
        b.set_equilibrium(i, 1.0, 0.0, 0.0, 1e-3, 201213487 + i)
    if tune:
        b.autotune(None, 3)
    ngroups = b.info(0).ngroups
    ms = time_steps(b.step, stream, steps, warmup)
    b.close()
    torch.cuda.synchronize()
    solvers = [make_solver(c, stream.cuda_stream) for c in cases]
    for i, s in enumerate(solvers):
        s.set_equilibrium(1.0, 0.0, 0.0, 1e-3, 201213487 + i)

    def loop(n):
        for _ in range(n):
            for s in solvers:
                s.step(1)

    ms_loop = time_steps(loop, stream, loop_steps, 1)
    for s in solvers:
        s.close()
    return {"value": dof * 5 * steps / (ms / 1e3), "loop_value": dof * 5 * loop_steps / (ms_loop / 1e3),
            "cases": len(cases), "groups": ngroups, "dof": dof, "steps": steps, "loop_steps": loop_steps,
            "ms_per_step": ms / steps, "loop_ms_per_step": ms_loop / loop_steps}


# ---------------------------------------------------------------- oracle timing
ORACLE_SAMPLE_SCRIPT = r"""
import json, sys, time
sys.path.insert(0, %(root)r)
import numpy as np
from oracle import dg
from paper_2012_13487_gb300 import inputs
w = json.loads(%(w)r)
kind, n = w["vel"]
if w["kind"] == "cavity":
    bc = ("diffuse",) * 4; wall = ((0, 0), (0, 0), (w["speed"], 0), (0, 0))
else:
    bc = ("diffuse", "periodic", "diffuse", "periodic"); wall = ((-w["speed"], 0), (0, 0), (w["speed"], 0), (0, 0))
mesh = inputs.unstructured_square(w["nx"], w["ny"], w["mesh_seed"], shuffle=False) if w.get("unstructured") else None
pr = dg.Problem(w["nx"], w["ny"], w["p"], velset=(kind, n), kn=w["kn"], bc=bc, wall_u=wall, mesh=mesh,
                nc_scale=np.sqrt(2.0) if w.get("nc_sqrt2") else 1.0)
f0 = pr.equilibrium_state(amp=1e-3, u=inputs.perturbation(1, pr.K, pr.Np, pr.Q))
rng = np.random.default_rng(0)
elems = np.sort(rng.choice(pr.K, min(pr.K, %(nelem)d), replace=False))
res = np.zeros((len(elems), pr.Np, pr.Q))
t_end = time.perf_counter() + %(seconds)f
stages = 0
t0 = time.perf_counter()
while stages < %(min_stages)d or time.perf_counter() < t_end:
    f1, res = pr.lsrk_stage(1, f0, res, elems)
    stages += 1
    if stages >= %(max_stages)d:
        break
dt = time.perf_counter() - t0
print(json.dumps({"dof_stages": stages * len(elems) * pr.Np * pr.Q, "seconds": dt, "stages": stages,
                  "elements": int(len(elems)), "K": int(pr.K)}))
"""


def oracle_sample(w, seconds, nelem=512, min_stages=1, max_stages=10 ** 9):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    script = ORACLE_SAMPLE_SCRIPT % dict(root=ROOT, w=json.dumps(w), seconds=seconds, nelem=nelem,
                                         min_stages=min_stages, max_stages=max_stages)
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_sample_all_cores(w, seconds, nelem=512):
    """The same oracle sample run by one single-threaded process per host core
    at once (each on its own element sample): the aggregate DOF-stage/s of all
    cores, as a CPU baseline that uses the whole host."""
    ncores = os.cpu_count() or 1
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    procs = []
    for c in range(ncores):
        script = ORACLE_SAMPLE_SCRIPT % dict(root=ROOT, w=json.dumps(w), seconds=seconds, nelem=nelem,
                                             min_stages=1, max_stages=10 ** 9)
        script = script.replace("default_rng(0)", "default_rng(%d)" % c)
        procs.append(subprocess.Popen([sys.executable, "-c", script], stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True, env=env))
    outs = []
    for pr in procs:
        o, e = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError("oracle sample failed: " + e[-2000:])
        outs.append(json.loads(o.strip().splitlines()[-1]))
    secs = max(o["seconds"] for o in outs)
    return {"dof_stages": sum(o["dof_stages"] for o in outs), "seconds": secs, "cores": ncores,
            "elements": outs[0]["elements"], "K": outs[0]["K"]}


ORACLE_ERROR_SCRIPT = r"""
import json, sys, time
sys.path.insert(0, %(root)r)
import numpy as np
from oracle import dg
from paper_2012_13487_gb300 import inputs
w = json.loads(%(w)r)
kind, n = w["vel"]
if w["kind"] == "cavity":
    bc = ("diffuse",) * 4; wall = ((0, 0), (0, 0), (w["speed"], 0), (0, 0))
else:
    bc = ("diffuse", "periodic", "diffuse", "periodic"); wall = ((-w["speed"], 0), (0, 0), (w["speed"], 0), (0, 0))
t0 = time.perf_counter()
mesh = inputs.unstructured_square(w["nx"], w["ny"], w["mesh_seed"], shuffle=False) if w.get("unstructured") else None
pr = dg.Problem(w["nx"], w["ny"], w["p"], velset=(kind, n), kn=w["kn"], bc=bc, wall_u=wall, mesh=mesh,
                nc_scale=np.sqrt(2.0) if w.get("nc_sqrt2") else 1.0)
f = pr.equilibrium_state(amp=%(amp)r, u=inputs.perturbation(%(seed)d, pr.K, pr.Np, pr.Q))
f = pr.run(f, %(steps)d)
orho, oux, ouy = pr.nodal_moments(f)
zero = lambda x, y: 0 * x
out = {"oracle_seconds": time.perf_counter() - t0}
for tag, path in json.loads(%(gpu)r).items():
    g = np.load(path)
    e_rho = pr.l2_error(g["rho"] - orho, zero)
    e_u = np.hypot(pr.l2_error(g["ux"] - oux, zero), pr.l2_error(g["uy"] - ouy, zero)) / w["speed"]
    out[tag] = {"l2_rho": float(e_rho), "l2_u_over_U": float(e_u),
                "max_abs_u_over_U": float(max(np.abs(g["ux"] - oux).max(), np.abs(g["uy"] - ouy).max()) / w["speed"]),
                "max_abs_rho": float(np.abs(g["rho"] - orho).max())}
print(json.dumps(out))
"""

ERROR_STEPS = 2
ERROR_AMP = 1e-3
ERROR_SEED = 201213487


def error_copy(w):
    """The mesh copy on which a workload's error against the FP64 oracle is
    taken: the workload itself when it has at most 32 x 32 cells, else its
    32 x 32 x 2 copy (the size the precision configuration names; 8 x 8 x 2 for
    more than 1024 velocities) with the same degree, velocity set, Kn and wall
    speed (and, for an unstructured workload, the same mesh generator)."""
    c = dict(w)
    cells = 32 if w["vel"][1] ** 2 <= 1024 else 8   # D2Q1089: an 8 x 8 x 2 copy
    c["nx"], c["ny"] = min(w["nx"], cells), min(w["ny"], cells)
    return c


def gpu_error_moments(w, forms, st, tmpdir):
    """Moments of each (precision, reduction) form after ERROR_STEPS steps on the
    error copy, from the seeded perturbed rest state drawn by the library."""
    import numpy as np
    import torch
    c = error_copy(w)
    paths = {}
    for form in forms:
        prec, red = form[0], form[1]
        rounding = form[2] if len(form) > 2 else 0
        wc = dict(c, precision=prec, reduction=red, rounding=rounding)
        s = make_solver(wc, st.cuda_stream)
        s.set_equilibrium(1.0, 0.0, 0.0, ERROR_AMP, ERROR_SEED)
        s.step(ERROR_STEPS)
        rho, ux, uy = s.moments()
        torch.cuda.synchronize()
        s.close()
        tag = "%s/%s" % (prec, red) + ("/stochastic" if rounding else "")
        path = os.path.join(tmpdir, tag.replace("/", "_") + ".npz")
        np.savez(path, rho=rho, ux=ux, uy=uy)
        paths[tag] = path
    return c, paths


def oracle_errors(c, paths):
    """L2 errors of rho and u (over the wall or lid speed) of the GPU forms
    against the FP64 oracle on the same copy and steps (oracle leg: a CPU
    subprocess with no GPU visible)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    script = ORACLE_ERROR_SCRIPT % dict(root=ROOT, w=json.dumps(c), amp=ERROR_AMP, seed=ERROR_SEED,
                                        steps=ERROR_STEPS, gpu=json.dumps(paths))
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle error run failed: " + r.stderr[-2000:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    out["copy"] = "%dx%dx2 triangles, p=%d, %s, Kn=%g, speed %g; %d LSRK(5,4) steps from the rest state " \
                  "x (1 + %g u), u SplitMix64 seed %d" % (c["nx"], c["ny"], c["p"], c["vel"], c["kn"], c["speed"],
                                                           ERROR_STEPS, ERROR_AMP, ERROR_SEED)
    return out


# ---------------------------------------------------------------- arms
def max_over_ranks(x, dist, device):
    """The largest x over all ranks (a job's time is its slowest rank's); x
    itself on one rank (dist None).  device: "cuda" for NCCL, "cpu" for gloo."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, seconds):
    """Whole-job units per second: every rank (a replica) processes
    units_per_rank in the slowest rank's time."""
    return world * units_per_rank / seconds


def pick_form(w, st, torch, steps=100):
    """Autotune the FMA form and, where the workload has one, the tensor-core
    form, time `steps` steps of each and keep the faster solver (the two are
    within a few per cent on some shapes, closer than the autotuner's short
    trials resolve)."""
    from paper_2012_13487_gb300 import fedbm as fb
    best, best_ms = None, None
    for tc in (-1, 1):
        try:
            s = make_solver(w, st.cuda_stream, tc=tc)
        except fb.FedbmError:
            continue            # no tensor-core form for this shape
        s.set_equilibrium(1.0, 0.0, 0.0, 0.0, 201213487)
        s.autotune(None, 20)
        s.step(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        s.step(steps)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if best_ms is None or ms < best_ms:
            if best is not None:
                best.close()
            best, best_ms = s, ms
        else:
            s.close()
    best.set_equilibrium(1.0, 0.0, 0.0, 0.0, 201213487)
    return best


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args, w, name):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    if w["kind"] == "batch":   # the oracle samples the first case of the batch
        w = dict(batch_case_list(w)[0], desc=w["desc"])
    K, Np, Q = dims(w)
    # each step: one LSRK stage of the oracle on 64 sampled elements (FP64)
    totals, seconds = 0, 0.0
    out = oracle_sample(w, seconds=0.0, nelem=64, min_stages=args.steps + args.warmup,
                        max_stages=args.steps + args.warmup)
    per_stage_s = out["seconds"] / out["stages"]
    dof_per_stage = out["dof_stages"] / out["stages"]
    value = dof_per_stage / per_stage_s
    line = {
        "impl": "reference", "metric": "DOF-stage updates/s", "value": value, "unit": "DOF-stage/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per_stage_s * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["desc"], "name": name, "K": K, "Np": Np, "Q": Q},
        "cpu_baseline": {"value": value, "unit": "DOF-stage/s", "cores": 1, "kind": "oracle",
                         "sample": "FP64 NumPy oracle, one LSRK stage per step on 64 sampled elements "
                                   "(%d DOF) of the %d-element mesh, single thread" % (dof_per_stage, K)},
        "e2e": {"value": value, "unit": "DOF-stage/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


REPEATS = 5
DTYPE = {"fp32": "f32", "fp64": "f64", "bf16": "bf16-state/f32", "fp16": "f16-state/f32"}


def timed_repeats(step, stream, steps, repeats, barrier, dist):
    """`repeats` timed regions of `steps` steps each: barrier + synchronize on
    both sides, CUDA events on the launching stream, the max over ranks of
    each region.  Returns the milliseconds of every region."""
    import torch
    out = []
    for _ in range(repeats):
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        out.append(max_over_ranks(e0.elapsed_time(e1), dist, "cuda"))
    return out


def spread(ms, steps):
    """Median and spread of repeated timed regions, per step."""
    per = [m / steps for m in ms]
    return {"n": len(per), "ms_per_step_median": statistics.median(per), "ms_per_step_min": min(per),
            "ms_per_step_max": max(per), "spread_pct": 100.0 * (max(per) - min(per)) / statistics.median(per)}


def kernel_name(info):
    """Name of the stage-kernel form a solver's configuration launches."""
    if info.tensor_cores:
        return "stage_kernel_tc"
    if info.velocity_split > 1:
        return "stage_kernel_cl"
    return "stage_kernel_ws" if info.pipeline_stages == 3 else "stage_kernel"


def roofline_of(dof, prec, ms_per_step, kernel, traffic=None):
    """Roofline of the stage kernel: algorithmic bytes of one launch over the
    average launch time (five launches per step, back to back in a graph)."""
    alg = dof * algorithmic_bytes_per_dof_step(prec)
    achieved = alg / (ms_per_step / 1e3) / 1e9
    peak, peak_kind = hbm_peak()
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": peak_kind, "traffic": traffic,
            "algorithmic_bytes_per_dof_step": algorithmic_bytes_per_dof_step(prec),
            "algorithmic_bytes_per_launch": alg / 5.0, "kernel": kernel}


def measure_form(w, st, steps, warmup, tune, repeats=3, profile=None):
    """Throughput of one (workload, precision, reduction) form: the FMA kernel
    by default, autotuned over both kernel forms when `tune`."""
    s = make_solver(w, st.cuda_stream)
    s.set_equilibrium(1.0, 0.0, 0.0, 0.0, 201213487)
    if tune:
        s.autotune(None, 10)
    K, Np, Q = dims(w)
    dof = K * Np * Q
    s.step(warmup)
    ms = timed_repeats(s.step, st, steps, repeats, lambda: None, None)
    sp = spread(ms, steps)
    info = s.info
    s.mass()
    s.close()
    kern = kernel_name(info)
    return {"value": dof * 5 / (sp["ms_per_step_median"] / 1e3), "unit": "DOF-stage/s", "workload": w["desc"],
            "precision": w["precision"], "reduction": w.get("reduction", "default"), "dof": dof,
            "steps": steps, "repeats": sp,
            "tile": {"elems_per_cta": info.elems_per_cta, "threads_per_cta": info.threads_per_cta,
                     "pipeline_stages": info.pipeline_stages, "grid": info.grid,
                     "tensor_cores": info.tensor_cores, "velocity_split": info.velocity_split},
            "roofline": roofline_of(dof, w["precision"], sp["ms_per_step_median"], kern,
                                    recorded_traffic(profile, kern, w["precision"]) if profile else None)}


def run_ours(args, w, name):
    import torch

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    st = torch.cuda.Stream()
    if w["kind"] == "batch":
        return run_batch_workload(args, w, name, st, world, rank, dist)
    K, Np, Q = dims(w)
    dof = K * Np * Q
    if not args.no_tune and not (args.epc or args.tpb or args.stages or args.tc):
        s = pick_form(w, st, torch)
    else:
        s = make_solver(w, st.cuda_stream, args.epc, args.tpb, args.stages, args.tc)
        s.set_equilibrium(1.0, 0.0, 0.0, 0.0, 201213487)
        if not args.no_tune and not (args.epc or args.tpb or args.stages or args.tc == 1):
            s.autotune(None, 20)
    s.step(args.warmup)
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()

    sampler = ClockSampler(local)
    sampler.start()
    ms_list = timed_repeats(s.step, st, args.steps, args.repeats, barrier, dist)
    clocks = sampler.stop()
    mass = s.mass()   # also raises on NaN / rho <= 0
    sp = spread(ms_list, args.steps)
    ms_step = sp["ms_per_step_median"]
    secs = ms_step * args.steps / 1e3
    value = job_throughput(world, dof * 5 * args.steps, secs)
    kern = kernel_name(s.info) + " (5 launches per step; average over the mix)"
    roof = roofline_of(dof, w["precision"], ms_step, kern,
                       recorded_traffic(name, kernel_name(s.info), w["precision"]))

    # end to end through the C ABI with host buffers
    e2e_steps = max(3, min(args.steps, 20))
    from paper_2012_13487_gb300 import fedbm as fb
    # the host state in the solver's natural input precision: FP64 for the FP64
    # form, FP32 (fedbm_set_state_f32) for the FP32 and 16-bit forms
    in_f32 = w["precision"] != "fp64"
    set_state = fb.fedbm_set_state_f32 if in_f32 else fb.fedbm_set_state
    in_dtype = torch.float32 if in_f32 else torch.float64
    s.set_equilibrium(1.0, 0.0, 0.0, 0.0, 201213487)
    f64 = torch.empty((K, Np, Q), dtype=torch.float64).pin_memory()
    fb.fedbm_get_state(s.h, f64, False)
    f_host = f64.to(in_dtype).pin_memory()
    del f64
    rho = torch.empty((K, Np), dtype=torch.float64).pin_memory()
    ux = torch.empty_like(rho).pin_memory()
    uy = torch.empty_like(rho).pin_memory()
    for _ in range(2):
        set_state(s.h, f_host, False)
        fb.fedbm_rk_step(s.h, 1)
        fb.fedbm_get_moments(s.h, rho, ux, uy, False)
    # (a) serial: the library's host path (copy into its staging buffer, encode,
    # step, read-out), one step after the other
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        set_state(s.h, f_host, False)
        fb.fedbm_rk_step(s.h, 1)
        fb.fedbm_get_moments(s.h, rho, ux, uy, False)
    torch.cuda.synchronize()
    serial_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    serial_value = job_throughput(world, dof * 5 * e2e_steps, serial_s)
    rho_serial = rho.clone()

    # (b) pipelined: step i+1's input crosses the host link on a copy stream
    # while step i is encoded, stepped and read out; every step's copy and
    # read-out stay inside the timed region
    cs = torch.cuda.Stream()
    d_in = [torch.empty((K, Np, Q), dtype=in_dtype, device="cuda") for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]

    def enqueue_copy(j):
        cs.wait_event(consumed[j])          # the encode that last read d_in[j]
        with torch.cuda.stream(cs):
            d_in[j].copy_(f_host, non_blocking=True)
        copied[j].record(cs)

    def pipelined(n):
        enqueue_copy(0)
        for i in range(n):
            j = i % 2
            if i + 1 < n:
                enqueue_copy((i + 1) % 2)
            st.wait_event(copied[j])
            set_state(s.h, d_in[j], True)
            consumed[j].record(st)
            fb.fedbm_rk_step(s.h, 1)
            fb.fedbm_get_moments(s.h, rho, ux, uy, False)

    pipelined(3)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pipelined(e2e_steps)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e_value = job_throughput(world, dof * 5 * e2e_steps, e2e_s)
    del d_in
    # every step starts from the same input, so the overlapped copies must
    # reproduce the serial read-out bit for bit
    if not torch.equal(rho, rho_serial):
        raise RuntimeError("pipelined end-to-end read-out differs from the serial one")
    tile = {"elems_per_cta": s.info.elems_per_cta, "threads_per_cta": s.info.threads_per_cta,
            "pipeline_stages": s.info.pipeline_stages, "grid": s.info.grid,
            "tensor_cores": s.info.tensor_cores}
    s.close()

    cpu = None
    error = None
    forms = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out = oracle_sample(w, seconds=args.cpu_seconds)
        cpu = {"value": out["dof_stages"] / out["seconds"], "unit": "DOF-stage/s", "cores": 1, "kind": "oracle",
               "sample": "FP64 NumPy oracle, %d LSRK stages on %d sampled elements (%d DOF each) of the "
                         "%d-element mesh, single thread, %.1f s" % (out["stages"], out["elements"],
                                                                     out["dof_stages"] // out["stages"],
                                                                     out["K"], out["seconds"])}
        allc = oracle_sample_all_cores(w, seconds=min(args.cpu_seconds, 10.0))
        cpu["all_cores"] = {"value": allc["dof_stages"] / allc["seconds"], "unit": "DOF-stage/s",
                            "cores": allc["cores"], "kind": "oracle",
                            "sample": "the same sample, one single-threaded oracle process per host core at "
                                      "once, each on %d sampled elements of its own" % allc["elements"]}
    if rank == 0 and world == 1 and not args.no_error:
        with tempfile.TemporaryDirectory() as td:
            copy, paths = gpu_error_moments(w, [(w["precision"], w.get("reduction", "default"))], st, td)
            error = oracle_errors(copy, paths)
    if rank == 0 and world == 1 and not args.no_forms and name == DEFAULT_WORKLOAD:
        forms = measure_forms(args, w, st, value, roof, error)
    if rank == 0:
        line = {
            "metric": "DOF-stage updates/s", "value": value, "unit": "DOF-stage/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[w["precision"]], "data": "synthetic",
            "config": {"workload": w["desc"], "name": name, "K": K, "Np": Np, "Q": Q, "dof": dof,
                       "reduction": w.get("reduction", "default"), "tile": tile,
                       "l2": "inputs larger than L2 (state x2 + residual = %.0f MB), no flush" %
                             (dof * (2 * STATE_BYTES[w["precision"]] + RES_BYTES[w["precision"]]) / 1e6),
                       "parallelism": "replicas x%d" % world},
            "repeats": sp,
            "roofline": roof,
            "error": error,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "DOF-stage/s", "steps": e2e_steps,
                    "h2d_bytes_per_step": dof * (4 if in_f32 else 8), "d2h_bytes_per_step": 3 * K * Np * 8,
                    "input_dtype": "f32" if in_f32 else "f64",
                    "path": "pinned host %s state -> device buffer on a copy stream (step i+1's copy overlaps "
                            "step i) + %s(device) + fedbm_rk_step(1) + fedbm_get_moments(host, FP64)"
                            % ("FP32" if in_f32 else "FP64", set_state.__name__),
                    "serial": {"value": serial_value, "unit": "DOF-stage/s",
                               "path": "%s(host) + fedbm_rk_step(1) + fedbm_get_moments(host), "
                                       "one step after the other" % set_state.__name__}},
            "gpu_launches": 5 * args.steps * args.repeats,
            "clocks": clocks,
            "mass_after": mass,
            "forms": forms,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# the other forms of the metric, each with its own roofline and error against
# the oracle: (key, workload, precision, reduction)
FORMS = [
    ("fp32_red_fp64", DEFAULT_WORKLOAD, "fp32", "fp64"),
    ("fp32_red_comp", DEFAULT_WORKLOAD, "fp32", "comp"),
    ("bf16_state", DEFAULT_WORKLOAD, "bf16", "default"),
    ("cavity_kn2_64x64x2_p4_nc16_fp32", "cavity_kn2_64x64x2_p4_nc16x16_fp32", "fp32", "default"),
    ("couette_256x256x2_p5_gh16_fp32", "couette_kn1_256x256x2_p5_gh16_fp32", "fp32", "default"),
    ("couette_256x256x2_p5_gh16_bf16", "couette_kn1_256x256x2_p5_gh16_bf16", "bf16", "default"),
    ("cavity_kn8_128x128x2_p3_nc32_bf16_red_fp64", "cavity_kn8_128x128x2_p3_nc32x32_bf16", "bf16", "fp64"),
    ("cavity_kn8_128x128x2_p3_nc32_bf16_red_comp", "cavity_kn8_128x128x2_p3_nc32x32_bf16", "bf16", "comp"),
    ("cavity_kn8_128x128x2_p3_nc32_fp16_red_fp64", "cavity_kn8_128x128x2_p3_nc32x32_bf16", "fp16", "fp64"),
    ("cavity_kn8_128x128x2_p3_nc32_fp32", "cavity_kn8_128x128x2_p3_nc32x32_bf16", "fp32", "default"),
    ("cavity_kn8_128x128x2_p3_nc32_fp32_red_comp", "cavity_kn8_128x128x2_p3_nc32x32_bf16", "fp32", "comp"),
    ("cavity_kn8_128x128x2_p3_nc32_bf16_stochastic", "cavity_kn8_128x128x2_p3_nc32x32_bf16", "bf16", "comp"),
    ("cavity_unstructured_8192_p4_nc16_fp32", "cavity_kn1_unstructured_8192_p4_nc16x16_fp32", "fp32", "default"),
    ("cavity_kn8_32x32x2_p5_d2q1089_fp32_split", "cavity_kn8_32x32x2_p5_nc33x33_sqrt2_fp32", "fp32", "default"),
]


# the committed ncu summary (by workload name) whose traffic a form reports
FORM_PROFILES = {
    "bf16_state": "cavity_kn1_64x64x2_p4_nc16x16_bf16",
    "couette_256x256x2_p5_gh16_fp32": "couette_kn1_256x256x2_p5_gh16_fp32",
    "cavity_kn8_128x128x2_p3_nc32_bf16_red_comp": "cavity_kn8_128x128x2_p3_nc32x32_bf16",
    "cavity_kn8_32x32x2_p5_d2q1089_fp32_split": "cavity_kn8_32x32x2_p5_nc33x33_sqrt2_fp32",
}


def measure_forms(args, w, st, value, roof, error):
    """Every form of FORMS (throughput, roofline, error on its copy) and the
    seeded 256-case batch against a loop of single solvers."""
    forms = {"fp32": {"value": value, "workload": w["desc"], "roofline": roof, "error": error},
             "unit": "DOF-stage/s"}
    steps = max(20, args.steps)
    by_copy = {}
    for key, wname, prec, red in FORMS:
        wf = dict(WORKLOADS[wname], precision=prec, reduction=red)
        if key.endswith("_stochastic"):
            wf["rounding"] = 1
        base = WORKLOADS[wname]["desc"].split(", BF16")[0].split(", FP32")[0]
        wf["desc"] = "%s [%s state, %s moment sums%s]" % (base, prec.upper(), red,
                                                         ", stochastic rounding" if wf.get("rounding") else "")
        forms[key] = measure_form(wf, st, steps, args.warmup, not args.no_tune, profile=FORM_PROFILES.get(key))
        by_copy.setdefault(wname, []).append((key, prec, red, wf.get("rounding", 0)))
    if not args.no_error:
        for wname, items in by_copy.items():
            wf = WORKLOADS[wname]
            with tempfile.TemporaryDirectory() as td:
                copy, paths = gpu_error_moments(wf, [(p, r, sr) for _, p, r, sr in items], st, td)
                errs = oracle_errors(copy, paths)
            for key, prec, red, sr in items:
                tag = "%s/%s" % (prec, red) + ("/stochastic" if sr else "")
                forms[key]["error"] = dict(errs[tag], copy=errs["copy"])
    bat = measure_batch(WORKLOADS["batch256_couette_cavity_fp32"], st, 10, 3, 2, not args.no_tune)
    forms["batched"] = dict(bat, workload=WORKLOADS["batch256_couette_cavity_fp32"]["desc"])
    forms["implicit_backward_euler"] = measure_implicit(st)
    return forms


def measure_implicit(st):
    """The implicit path: backward-Euler steps (Newton with matrix-free GMRES,
    every residual one fused stage-kernel launch) of a Couette case; reported
    as residual evaluations x DOF per second and time per step."""
    import torch
    from paper_2012_13487_gb300 import fedbm as fb
    w = dict(kind="couette", nx=16, ny=16, p=3, vel=("gh", 4), kn=1.0, speed=0.1, precision="fp64")
    K, Np, Q = dims(w)
    out = {}
    for pc in (1, 0):
        s = make_solver(w, st.cuda_stream)
        s.set_equilibrium(1.0, 0.0, 0.0, 1e-3, 201213487)
        ip = fb.implicit_params(fb.IMPLICIT_BE, 0.5, newton_rtol=1e-8, newton_atol=1e-12, gmres_rtol=1e-3,
                                gmres_restart=40, gmres_max_iter=4000, preconditioner=pc)
        s.implicit_step(ip, 1)            # warm-up (work space, preconditioner, first launches)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        stats = s.implicit_step(ip, 3)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        s.close()
        out["block_jacobi" if pc else "no_preconditioner"] = {
            "value": stats.rhs_evals * K * Np * Q / secs, "unit": "DOF-residual evaluations/s",
            "s_per_step": secs / 3, "newton_iters": stats.newton_iters, "gmres_iters": stats.gmres_iters,
            "rhs_evals": stats.rhs_evals, "converged": bool(stats.converged)}
    out["workload"] = ("Couette Kn=1, 16x16x2 triangles, p=3, GH D2Q16, FP64; backward Euler dt = 0.5, 3 steps, "
                       "Newton to 1e-8 relative, GMRES(40) forcing 1e-3")
    return out


def run_batch_workload(args, w, name, st, world, rank, dist):
    """The seeded 256-case batch as the timed workload (one graph launch per
    step advances every case); the case-by-case loop is reported beside it."""
    import torch
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    if dist is not None:
        dist.barrier()
    bat = measure_batch(w, st, args.steps, args.warmup, max(1, min(args.steps, 3)), not args.no_tune)
    clocks = sampler.stop()
    ms = max_over_ranks(bat["ms_per_step"] * args.steps, dist, "cuda")
    value = job_throughput(world, bat["dof"] * 5 * args.steps, ms / 1e3)
    peak, peak_kind = hbm_peak()
    achieved = bat["dof"] * algorithmic_bytes_per_dof_step("fp32") * args.steps / (ms / 1e3) / 1e9
    if rank == 0:
        line = {
            "metric": "DOF-stage updates/s", "value": value, "unit": "DOF-stage/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w["desc"], "name": name, "cases": bat["cases"], "groups": bat["groups"],
                       "dof": bat["dof"], "l2": "inputs larger than L2, no flush",
                       "parallelism": "replicas x%d" % world},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_kind, "traffic": None,
                         "algorithmic_bytes_per_dof_step": algorithmic_bytes_per_dof_step("fp32"),
                         "kernel": "stage_kernel, all groups"},
            "loop_baseline": {"value": bat["loop_value"], "unit": "DOF-stage/s",
                              "ms_per_step": bat["loop_ms_per_step"],
                              "what": "the same cases stepped one solver at a time"},
            "cpu_baseline": None,
            "e2e": None,
            "gpu_launches": 5 * bat["groups"] * args.steps,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--epc", type=int, default=0, help="stage tile: elements per CTA (0 = library default)")
    ap.add_argument("--tpb", type=int, default=0, help="stage tile: threads per CTA (0 = library default)")
    ap.add_argument("--stages", type=int, default=0, help="stage tile buffers per CTA (0 = library default)")
    ap.add_argument("--tc", type=int, default=0, choices=[-1, 0, 1],
                    help="stage-kernel form: 1 tensor cores, -1 FMA only, 0 library default")
    ap.add_argument("--no-tune", action="store_true", help="skip the tile autotuner")
    ap.add_argument("--no-forms", action="store_true", help="skip the other forms (precisions, reductions, "
                    "the p=5 Couette and Kn=8 cavity configurations, the batch)")
    ap.add_argument("--no-error", action="store_true", help="skip the error against the oracle")
    ap.add_argument("--repeats", type=int, default=REPEATS, help="timed regions of --steps steps (median reported)")
    ap.add_argument("--reduction", default=None, choices=sorted(RED), help="moment sums (default: the workload's)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    w = WORKLOADS[args.workload]
    if args.reduction:
        w = dict(w, reduction=args.reduction)
    if args.impl == "reference":
        run_reference(args, w, args.workload)
    else:
        run_ours(args, w, args.workload)


if __name__ == "__main__":
    main()
