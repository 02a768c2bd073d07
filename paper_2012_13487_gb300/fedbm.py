"""ctypes binding of ``libfedbm.so`` (C ABI in ``include/fedbm.h``).

Argument marshalling only: every function here forwards to the C entry point
of the same name; all computation runs in the CUDA library.  PyTorch is used
only to supply device buffers and streams (``tensor.data_ptr()``,
``torch.cuda.current_stream().cuda_stream``).  Loading fails loudly if the
library has not been built.
"""
import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libfedbm.so")

FEDBM_OK = 0
FEDBM_EINVAL = -1
FEDBM_ENOMEM = -2
FEDBM_ECUDA = -3
FEDBM_ENONFINITE = -4
FEDBM_ETIMEOUT = -5
FEDBM_ENOTSUP = -6

BC_PERIODIC, BC_WALL_DIFFUSE, BC_WALL_EQ = 0, 1, 2
VELSET_GH, VELSET_NC = 0, 1
FP64, FP32, BF16_DEV, FP16_DEV = 0, 1, 2, 3
RED_DEFAULT, RED_FP64, RED_COMP_FP32 = 0, 1, 2
TAU_KN, TAU_KIM_PITSCH, TAU_PSI = 0, 1, 2


class MeshDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("order", ctypes.c_int32),
                ("bc", ctypes.c_int32 * 4), ("wall_ux", ctypes.c_double * 4),
                ("wall_uy", ctypes.c_double * 4), ("lx", ctypes.c_double), ("ly", ctypes.c_double),
                ("nvert", ctypes.c_int32), ("ntri", ctypes.c_int32),
                ("vert_xy", ctypes.c_void_p), ("tri", ctypes.c_void_p)]


class VelsetDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n", ctypes.c_int32), ("nc_extent", ctypes.c_double),
                ("nc_sqrt2", ctypes.c_int32), ("eq_order", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("kn", ctypes.c_double), ("length", ctypes.c_double), ("beta", ctypes.c_double),
                ("cfl", ctypes.c_double), ("dt", ctypes.c_double), ("precision", ctypes.c_int32),
                ("reduction", ctypes.c_int32), ("collision", ctypes.c_int32),
                ("elems_per_cta", ctypes.c_int32), ("threads_per_cta", ctypes.c_int32),
                ("pipeline_stages", ctypes.c_int32), ("tensor_cores", ctypes.c_int32),
                ("test_wait_timeout", ctypes.c_int32), ("tau_model", ctypes.c_int32),
                ("velocity_split", ctypes.c_int32), ("rounding", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int64), ("Np", ctypes.c_int64), ("Nfp", ctypes.c_int64),
                ("Q", ctypes.c_int64), ("Q_padded", ctypes.c_int64), ("dt", ctypes.c_double),
                ("tau", ctypes.c_double), ("time", ctypes.c_double), ("steps", ctypes.c_int64),
                ("precision", ctypes.c_int32), ("reduction", ctypes.c_int32), ("order", ctypes.c_int32),
                ("eq_order", ctypes.c_int32), ("elems_per_cta", ctypes.c_int32),
                ("threads_per_cta", ctypes.c_int32), ("pipeline_stages", ctypes.c_int32),
                ("grid", ctypes.c_int32), ("group", ctypes.c_int32), ("ngroups", ctypes.c_int32),
                ("tensor_cores", ctypes.c_int32), ("velocity_split", ctypes.c_int32),
                ("state_bytes", ctypes.c_int64),
                ("residual_bytes", ctypes.c_int64)]


IMPLICIT_BE, IMPLICIT_SDIRK3_O4, IMPLICIT_SDIRK5_O4, IMPLICIT_CUSTOM = 0, 1, 2, 3
FEDBM_ENOCONV = -7


class ImplicitParams(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int32), ("stages", ctypes.c_int32), ("A", ctypes.c_double * 36),
                ("b", ctypes.c_double * 6), ("dt", ctypes.c_double), ("newton_rtol", ctypes.c_double),
                ("newton_atol", ctypes.c_double), ("newton_max_iter", ctypes.c_int32),
                ("gmres_restart", ctypes.c_int32), ("gmres_max_iter", ctypes.c_int32),
                ("gmres_rtol", ctypes.c_double), ("preconditioner", ctypes.c_int32)]


class ImplicitStats(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int32), ("gmres_iters", ctypes.c_int32), ("rhs_evals", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("residual", ctypes.c_double)]


class CaseDesc(ctypes.Structure):
    _fields_ = [("mesh", MeshDesc), ("velset", VelsetDesc), ("params", Params)]


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)

# name -> (restype, argtypes); exactly the entry points of include/fedbm.h
SIGNATURES = {
    "fedbm_velset": (ctypes.c_int, [ctypes.POINTER(VelsetDesc), _P, _P, _P, _I32]),
    "fedbm_ref_operators": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _P, _P, _P, _P]),
    "fedbm_mesh_nodes": (ctypes.c_int, [ctypes.POINTER(MeshDesc), ctypes.POINTER(VelsetDesc),
                                        ctypes.POINTER(Params), _P, _P, _D]),
    "fedbm_mesh_connectivity": (ctypes.c_int, [ctypes.POINTER(MeshDesc), _P]),
    "fedbm_create": (ctypes.c_int, [ctypes.POINTER(MeshDesc), ctypes.POINTER(VelsetDesc),
                                    ctypes.POINTER(Params), _P, ctypes.POINTER(_P)]),
    "fedbm_destroy": (None, [_P]),
    "fedbm_set_state": (ctypes.c_int, [_P, _P, ctypes.c_int32]),
    "fedbm_set_state_f32": (ctypes.c_int, [_P, _P, ctypes.c_int32]),
    "fedbm_batch_set_state_f32": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32]),
    "fedbm_set_equilibrium": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_uint64]),
    "fedbm_rk_step": (ctypes.c_int, [_P, ctypes.c_int32]),
    "fedbm_rk_stage": (ctypes.c_int, [_P, ctypes.c_int32]),
    "fedbm_implicit_step": (ctypes.c_int, [_P, ctypes.POINTER(ImplicitParams), ctypes.c_int32,
                                           ctypes.POINTER(ImplicitStats)]),
    "fedbm_get_moments": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int32]),
    "fedbm_get_state": (ctypes.c_int, [_P, _P, ctypes.c_int32]),
    "fedbm_get_residual": (ctypes.c_int, [_P, _P, ctypes.c_int32]),
    "fedbm_mass": (ctypes.c_int, [_P, _D]),
    "fedbm_info": (ctypes.c_int, [_P, ctypes.POINTER(Info)]),
    "fedbm_last_error": (ctypes.c_char_p, []),
    "fedbm_mass_noalloc": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                          _P, _P, _P]),
    "fedbm_batch_create": (ctypes.c_int, [ctypes.POINTER(CaseDesc), ctypes.c_int32, _P, ctypes.POINTER(_P)]),
    "fedbm_batch_destroy": (None, [_P]),
    "fedbm_batch_set_state": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32]),
    "fedbm_batch_set_equilibrium": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                                   ctypes.c_double, ctypes.c_double, ctypes.c_uint64]),
    "fedbm_batch_get_state": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32]),
    "fedbm_batch_get_moments": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, ctypes.c_int32]),
    "fedbm_batch_mass": (ctypes.c_int, [_P, ctypes.c_int32, _D]),
    "fedbm_batch_info": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(Info)]),
    "fedbm_batch_rk_step": (ctypes.c_int, [_P, ctypes.c_int32]),
    "fedbm_batch_set_tiles": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "fedbm_batch_set_tensor_cores": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    "fedbm_batch_autotune": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.c_int32]),
    "fedbm_autotune": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.c_int32]),
}

_lib = None


def lib():
    """Load libfedbm.so once; raise if it is missing (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError("libfedbm.so is not built (run __graft_entry__.build() or "
                               "python -m paper_2012_13487_gb300.build)")
        L = ctypes.CDLL(_LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class FedbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("fedbm error %d: %s" % (code, msg))
        self.code = code


def _check(rc):
    if rc != FEDBM_OK:
        raise FedbmError(rc, lib().fedbm_last_error().decode())
    return rc


def _ptr(a):
    """Pointer of a NumPy array or a torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()


# ---- descriptor helpers ------------------------------------------------------
def mesh_desc(nx, ny, order, bc=(BC_WALL_DIFFUSE, BC_PERIODIC, BC_WALL_DIFFUSE, BC_PERIODIC),
              wall_u=((0, 0), (0, 0), (0, 0), (0, 0)), lx=1.0, ly=1.0):
    d = MeshDesc()
    d.nx, d.ny, d.order = nx, ny, order
    for s in range(4):
        d.bc[s] = bc[s]
        d.wall_ux[s] = wall_u[s][0]
        d.wall_uy[s] = wall_u[s][1]
    d.lx, d.ly = lx, ly
    return d


def unstructured_mesh_desc(vert_xy, tri, order, bc=(BC_WALL_DIFFUSE,) * 4,
                           wall_u=((0, 0), (0, 0), (0, 0), (0, 0))):
    """Descriptor of a conforming triangulation (vertices [nv][2], counter-
    clockwise triangles [nt][3]).  The arrays are kept alive on the returned
    descriptor (attribute ``_keep``) because the C side reads them when the
    descriptor is used."""
    v = np.ascontiguousarray(vert_xy, dtype=np.float64)
    t = np.ascontiguousarray(tri, dtype=np.int32)
    assert v.ndim == 2 and v.shape[1] == 2 and t.ndim == 2 and t.shape[1] == 3
    d = mesh_desc(0, 0, order, bc=bc, wall_u=wall_u, lx=0.0, ly=0.0)
    d.nvert, d.ntri = v.shape[0], t.shape[0]
    d.vert_xy, d.tri = v.ctypes.data, t.ctypes.data
    d._keep = (v, t)
    return d


def velset_desc(kind=VELSET_GH, n=4, eq_order=2, nc_extent=4.0, nc_sqrt2=0):
    d = VelsetDesc()
    d.kind, d.n, d.eq_order, d.nc_extent, d.nc_sqrt2 = kind, n, eq_order, nc_extent, nc_sqrt2
    return d


def params(kn=1.0, precision=FP32, reduction=RED_DEFAULT, cfl=0.5, dt=0.0, beta=1.0, collision=1,
           length=1.0, elems_per_cta=0, threads_per_cta=0, pipeline_stages=0, tensor_cores=0,
           test_wait_timeout=0, tau_model=0, velocity_split=0, rounding=0):
    p = Params()
    p.kn, p.length, p.beta, p.cfl, p.dt = kn, length, beta, cfl, dt
    p.precision, p.reduction, p.collision = precision, reduction, collision
    p.elems_per_cta, p.threads_per_cta = elems_per_cta, threads_per_cta
    p.pipeline_stages = pipeline_stages
    p.tensor_cores = tensor_cores
    p.test_wait_timeout = test_wait_timeout
    p.tau_model = tau_model
    p.velocity_split = velocity_split
    p.rounding = rounding
    return p


# ---- entry points (same names as the C ABI) ----------------------------------
def fedbm_velset(vs):
    q = ctypes.c_int32()
    _check(lib().fedbm_velset(ctypes.byref(vs), None, None, None, ctypes.byref(q)))
    ex, ey, w = (np.zeros(q.value) for _ in range(3))
    _check(lib().fedbm_velset(ctypes.byref(vs), _ptr(ex), _ptr(ey), _ptr(w), ctypes.byref(q)))
    return ex, ey, w


def fedbm_ref_operators(p):
    Np, Nfp = (p + 1) * (p + 2) // 2, p + 1
    out = dict(r=np.zeros(Np), s=np.zeros(Np), Dr=np.zeros((Np, Np)), Ds=np.zeros((Np, Np)),
               LIFT=np.zeros((Np, 3 * Nfp)), M=np.zeros((Np, Np)), fmask=np.zeros((3, Nfp), np.int32))
    _check(lib().fedbm_ref_operators(p, *(_ptr(out[k]) for k in ("r", "s", "Dr", "Ds", "LIFT", "M", "fmask"))))
    return out


def mesh_elements(mesh):
    """Element count K of a mesh descriptor."""
    return mesh.ntri if mesh.ntri > 0 else 2 * mesh.nx * mesh.ny


def fedbm_mesh_nodes(mesh, vs=None, prm=None):
    K = mesh_elements(mesh)
    Np = (mesh.order + 1) * (mesh.order + 2) // 2
    x, y = np.zeros((K, Np)), np.zeros((K, Np))
    dt = ctypes.c_double(0.0)
    _check(lib().fedbm_mesh_nodes(ctypes.byref(mesh), ctypes.byref(vs) if vs else None,
                                  ctypes.byref(prm) if prm else None, _ptr(x), _ptr(y),
                                  ctypes.byref(dt) if (vs and prm) else None))
    return x, y, dt.value


def fedbm_mesh_connectivity(mesh):
    nbr = np.zeros((mesh_elements(mesh), 3), np.int32)
    _check(lib().fedbm_mesh_connectivity(ctypes.byref(mesh), _ptr(nbr)))
    return nbr


def fedbm_create(mesh, vs, prm, stream=0):
    h = ctypes.c_void_p()
    _check(lib().fedbm_create(ctypes.byref(mesh), ctypes.byref(vs), ctypes.byref(prm),
                              ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def fedbm_destroy(h):
    lib().fedbm_destroy(h)


def fedbm_set_state(h, f, on_device):
    _check(lib().fedbm_set_state(h, _ptr(f), int(on_device)))


def fedbm_set_state_f32(h, f, on_device):
    _check(lib().fedbm_set_state_f32(h, _ptr(f), int(on_device)))


def fedbm_batch_set_state_f32(h, c, f, on_device):
    _check(lib().fedbm_batch_set_state_f32(h, c, _ptr(f), int(on_device)))


def fedbm_set_equilibrium(h, rho0=1.0, ux0=0.0, uy0=0.0, amp=0.0, seed=0):
    _check(lib().fedbm_set_equilibrium(h, rho0, ux0, uy0, amp, seed))


def fedbm_rk_step(h, nsteps=1):
    _check(lib().fedbm_rk_step(h, nsteps))


def fedbm_rk_stage(h, stage):
    _check(lib().fedbm_rk_stage(h, stage))


def implicit_params(scheme=IMPLICIT_BE, dt=1.0, newton_rtol=0.0, newton_atol=0.0, newton_max_iter=0,
                    gmres_restart=0, gmres_max_iter=0, gmres_rtol=0.0, A=None, b=None, preconditioner=0):
    ip = ImplicitParams()
    ip.preconditioner = preconditioner
    ip.scheme, ip.dt = scheme, dt
    ip.newton_rtol, ip.newton_atol, ip.newton_max_iter = newton_rtol, newton_atol, newton_max_iter
    ip.gmres_restart, ip.gmres_max_iter, ip.gmres_rtol = gmres_restart, gmres_max_iter, gmres_rtol
    if A is not None:
        A = np.asarray(A, dtype=np.float64)
        ip.stages = A.shape[0]
        for i in range(A.shape[0]):
            for j in range(A.shape[1]):
                ip.A[6 * i + j] = A[i, j]
        for j, v in enumerate(b):
            ip.b[j] = v
    return ip


def fedbm_implicit_step(h, ip, nsteps=1):
    st = ImplicitStats()
    _check(lib().fedbm_implicit_step(h, ctypes.byref(ip), nsteps, ctypes.byref(st)))
    return st


def fedbm_get_moments(h, rho, ux, uy, on_device):
    _check(lib().fedbm_get_moments(h, _ptr(rho), _ptr(ux), _ptr(uy), int(on_device)))


def fedbm_get_state(h, f, on_device):
    _check(lib().fedbm_get_state(h, _ptr(f), int(on_device)))


def fedbm_get_residual(h, r, on_device):
    _check(lib().fedbm_get_residual(h, _ptr(r), int(on_device)))


def fedbm_mass(h):
    m = ctypes.c_double()
    _check(lib().fedbm_mass(h, ctypes.byref(m)))
    return m.value


def fedbm_info(h):
    info = Info()
    _check(lib().fedbm_info(h, ctypes.byref(info)))
    return info


def fedbm_mass_noalloc(f, jac, mass_colsum, K, Np, Q, total, status, stream=0):
    """Allocation-free mass diagnostic on caller-owned device buffers (see the C header)."""
    _check(lib().fedbm_mass_noalloc(_ptr(f), _ptr(jac), _ptr(mass_colsum), K, Np, Q, _ptr(total),
                                    _ptr(status), ctypes.c_void_p(stream)))


def fedbm_batch_create(cases, stream=0):
    arr = (CaseDesc * len(cases))(*cases)
    h = ctypes.c_void_p()
    _check(lib().fedbm_batch_create(arr, len(cases), ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def fedbm_batch_destroy(h):
    lib().fedbm_batch_destroy(h)


def fedbm_batch_set_state(h, c, f, on_device):
    _check(lib().fedbm_batch_set_state(h, c, _ptr(f), int(on_device)))


def fedbm_batch_set_equilibrium(h, c, rho0=1.0, ux0=0.0, uy0=0.0, amp=0.0, seed=0):
    _check(lib().fedbm_batch_set_equilibrium(h, c, rho0, ux0, uy0, amp, seed))


def fedbm_batch_get_state(h, c, f, on_device):
    _check(lib().fedbm_batch_get_state(h, c, _ptr(f), int(on_device)))


def fedbm_batch_get_moments(h, c, rho, ux, uy, on_device):
    _check(lib().fedbm_batch_get_moments(h, c, _ptr(rho), _ptr(ux), _ptr(uy), int(on_device)))


def fedbm_batch_mass(h, c):
    m = ctypes.c_double()
    _check(lib().fedbm_batch_mass(h, c, ctypes.byref(m)))
    return m.value


def fedbm_batch_info(h, c):
    info = Info()
    _check(lib().fedbm_batch_info(h, c, ctypes.byref(info)))
    return info


def fedbm_batch_rk_step(h, nsteps=1):
    _check(lib().fedbm_batch_rk_step(h, nsteps))


def fedbm_batch_set_tiles(h, group, elems_per_cta=0, threads_per_cta=0, pipeline_stages=0):
    _check(lib().fedbm_batch_set_tiles(h, group, elems_per_cta, threads_per_cta, pipeline_stages))


def fedbm_batch_set_tensor_cores(h, group, on=1):
    _check(lib().fedbm_batch_set_tensor_cores(h, group, on))


def fedbm_batch_autotune(h, cache_path=None, trials=0):
    _check(lib().fedbm_batch_autotune(h, cache_path.encode() if cache_path else None, trials))


def fedbm_autotune(h, cache_path=None, trials=0):
    _check(lib().fedbm_autotune(h, cache_path.encode() if cache_path else None, trials))


def case_desc(mesh, vs, prm):
    c = CaseDesc()
    c.mesh, c.velset, c.params = mesh, vs, prm
    c._keep = getattr(mesh, "_keep", None)   # an unstructured mesh's arrays
    return c


class Batch:
    """Owning handle of a batch of cases."""

    def __init__(self, cases, stream=0):
        self.h = fedbm_batch_create(cases, stream)
        self.n = len(cases)

    def info(self, c):
        return fedbm_batch_info(self.h, c)

    def shape(self, c):
        i = fedbm_batch_info(self.h, c)
        return (i.K, i.Np, i.Q)

    def set_state(self, c, f, on_device=False):
        fedbm_batch_set_state(self.h, c, f, on_device)

    def set_equilibrium(self, c, rho0=1.0, ux0=0.0, uy0=0.0, amp=0.0, seed=0):
        fedbm_batch_set_equilibrium(self.h, c, rho0, ux0, uy0, amp, seed)

    def step(self, n=1):
        fedbm_batch_rk_step(self.h, n)

    def state(self, c):
        f = np.zeros(self.shape(c))
        fedbm_batch_get_state(self.h, c, f, False)
        return f

    def moments(self, c):
        K, Np, _ = self.shape(c)
        rho, ux, uy = np.zeros((K, Np)), np.zeros((K, Np)), np.zeros((K, Np))
        fedbm_batch_get_moments(self.h, c, rho, ux, uy, False)
        return rho, ux, uy

    def mass(self, c):
        return fedbm_batch_mass(self.h, c)

    def autotune(self, cache_path=None, trials=0):
        fedbm_batch_autotune(self.h, cache_path, trials)

    def set_tensor_cores(self, group, on=1):
        """Switch one kernel group to the tensor-core form (on=1) or back to the
        FMA form with automatic tiles (on=0)."""
        fedbm_batch_set_tensor_cores(self.h, group, on)

    def close(self):
        if self.h is not None and self.h.value:
            fedbm_batch_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """Owning handle: create on construction, destroy on close/garbage collection."""

    def __init__(self, mesh, vs, prm, stream=0):
        self.h = fedbm_create(mesh, vs, prm, stream)

    @property
    def info(self):
        """fedbm_info of the solver now (tile, time step, time, steps, ...)."""
        return fedbm_info(self.h)

    @property
    def shape(self):
        i = fedbm_info(self.h)
        return (i.K, i.Np, i.Q)

    def set_state(self, f, on_device=False):
        fedbm_set_state(self.h, f, on_device)

    def set_equilibrium(self, rho0=1.0, ux0=0.0, uy0=0.0, amp=0.0, seed=0):
        fedbm_set_equilibrium(self.h, rho0, ux0, uy0, amp, seed)

    def step(self, n=1):
        fedbm_rk_step(self.h, n)

    def stage(self, s):
        fedbm_rk_stage(self.h, s)

    def implicit_step(self, ip, n=1):
        """n implicit SDIRK steps (Newton-GMRES); returns the ImplicitStats."""
        return fedbm_implicit_step(self.h, ip, n)

    def state(self):
        f = np.zeros(self.shape)
        fedbm_get_state(self.h, f, False)
        return f

    def residual(self):
        r = np.zeros(self.shape)
        fedbm_get_residual(self.h, r, False)
        return r

    def moments(self):
        K, Np, _ = self.shape
        rho, ux, uy = np.zeros((K, Np)), np.zeros((K, Np)), np.zeros((K, Np))
        fedbm_get_moments(self.h, rho, ux, uy, False)
        return rho, ux, uy

    def mass(self):
        return fedbm_mass(self.h)

    def autotune(self, cache_path=None, trials=0):
        fedbm_autotune(self.h, cache_path, trials)

    def close(self):
        if self.h is not None and self.h.value:
            fedbm_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
