"""Test cases: one description builds both the oracle problem and the CUDA solver."""
import numpy as np

from oracle import dg
from paper_2012_13487_gb300 import inputs

BC_CODE = {"periodic": 0, "diffuse": 1, "eq": 2}
PREC_CODE = {"fp64": 0, "fp32": 1, "bf16": 2, "fp16": 3}
RED_CODE = {"default": 0, "fp64": 1, "comp": 2}
TAU_CODE = {"kn": 0, "kim_pitsch": 1, "psi": 2}

COUETTE_BC = ("diffuse", "periodic", "diffuse", "periodic")
CAVITY_BC = ("diffuse",) * 4


def couette(nx, ny, p, U=0.1, **kw):
    return dict(nx=nx, ny=ny, p=p, bc=COUETTE_BC, wall_u=((-U, 0), (0, 0), (U, 0), (0, 0)), **kw)


def cavity(nx, ny, p, U=0.1, **kw):
    return dict(nx=nx, ny=ny, p=p, bc=CAVITY_BC, wall_u=((0, 0), (0, 0), (U, 0), (0, 0)), **kw)


def unstructured(c, nx, ny, seed=11, shuffle=True):
    """Case c on a seeded unstructured triangulation of the unit square with
    about as many cells (2 nx ny triangles)."""
    return dict(c, mesh=inputs.unstructured_square(nx, ny, seed, shuffle=shuffle))


def oracle_problem(c):
    vs = c.get("velset", ("gh", 4))
    return dg.Problem(c["nx"], c["ny"], c["p"], velset=vs, eq_order=c.get("eq_order", 2),
                      kn=c.get("kn", 1.0), beta=c.get("beta", 1.0), bc=c["bc"], wall_u=c["wall_u"],
                      cfl=c.get("cfl", 0.5), collision=c.get("collision", True),
                      nc_scale=np.sqrt(2.0) if c.get("nc_sqrt2", False) else 1.0, mesh=c.get("mesh"),
                      tau_model=c.get("tau_model", "kn"))


def descriptors(c, precision="fp32", reduction="default", **tile):
    """(mesh, velset, params) descriptors of a case dict for the C ABI."""
    from paper_2012_13487_gb300 import fedbm as fb
    vs = c.get("velset", ("gh", 4))
    if c.get("mesh") is not None:
        m = fb.unstructured_mesh_desc(c["mesh"][0], c["mesh"][1], c["p"], bc=tuple(BC_CODE[b] for b in c["bc"]),
                                      wall_u=c["wall_u"])
    else:
        m = fb.mesh_desc(c["nx"], c["ny"], c["p"], bc=tuple(BC_CODE[b] for b in c["bc"]), wall_u=c["wall_u"])
    v = fb.velset_desc(fb.VELSET_GH if vs[0] == "gh" else fb.VELSET_NC, vs[1], c.get("eq_order", 2),
                       nc_sqrt2=int(c.get("nc_sqrt2", False)))
    prm = fb.params(kn=c.get("kn", 1.0), precision=PREC_CODE[precision], reduction=RED_CODE[reduction],
                    cfl=c.get("cfl", 0.5), beta=c.get("beta", 1.0), collision=int(c.get("collision", True)),
                    elems_per_cta=tile.get("epc", 0), threads_per_cta=tile.get("tpb", 0),
                    pipeline_stages=tile.get("stages", 0), tensor_cores=tile.get("tc", 0),
                    test_wait_timeout=tile.get("test_wait_timeout", 0),
                    tau_model=TAU_CODE[c.get("tau_model", "kn")], velocity_split=tile.get("vsplit", 0),
                    rounding=tile.get("rounding", 0))
    return m, v, prm


def solver(c, precision="fp32", reduction="default", **tile):
    from paper_2012_13487_gb300 import fedbm as fb
    return fb.Solver(*descriptors(c, precision, reduction, **tile))


def batch(cs, precision="fp32", reduction="default", **tile):
    from paper_2012_13487_gb300 import fedbm as fb
    return fb.Batch([fb.case_desc(*descriptors(c, precision, reduction, **tile)) for c in cs])


def initial_state(pr, amp=1e-3, seed=201213487, rho0=1.0, ux0=0.0, uy0=0.0):
    u = inputs.perturbation(seed, pr.K, pr.Np, pr.Q)
    return pr.equilibrium_state(rho0, ux0, uy0, amp, u)


def rel_max_err(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())
