"""DG discretisation of the discrete-velocity BGK equation, FP64.  Test
infrastructure only.

Follows Sec. II of the paper step by step:

* moments rho = sum_i f_i, rho u = sum_i e_i f_i                (Sec. II.A.2)
* Hermite equilibrium f_i^eq = w_i rho [1 + e.u + ((e.u)^2 - u^2)/2]
  (eq. feq, theta = RT = 1); with eq_order = 3 the third Hermite term of
  eq. Herm3a, w_i rho [(e.u)^3/6 - (e.u) u^2/2], is added
* tau = Kn L / (sqrt(3) c_s), c_s = 1                           (eq. KnTau)
* residual: the strong form of eq. byparts,
      df_i/dt = -(e_i . grad) f_i
                + M^-1 oint phi (F_i^- - F_i^*) . n ds
                - (f_i - f_i^eq) / tau,
  which equals eq. byparts because e_i f_i is a degree-p polynomial on a
  straight-sided triangle (all integrals exact); the nonlinear f^eq enters
  by nodal collocation (the paper does not say how it is projected).
* numerical flux F^* . n = (e.n){{f}} + (2 beta - 1) |e.n| (f^- - f^+)/2,
  i.e. upwind for beta = 1 and central for beta = 1/2 (Sec. II.B.1; the
  printed form with [[f]] is read as the standard upwind/central family);
  so (F^- - F^*).n = ((e.n) - (2beta-1)|e.n|)/2 * (f^- - f^+).
* walls (Sec. II.B.2): the exterior state of an incoming velocity
  (e_i . n < 0) is the diffuse-scattering value of eq. FullBC,
      f_i^+ = rho_w f_i^eq(1, u_b),
      rho_w = sum_{e_j.n > 0} (e_j.n) f_j^- / sum_{e_k.n < 0} |e_k.n| f_k^eq(1, u_b),
  or f_i^eq(1, u_b) for eq. UsedBC ("eq" walls, rho_b = 1).  Walls move
  tangentially (u_b . n = 0), so (e - u_b) . n = e . n.  Outgoing
  velocities take f^+ = f^- (no jump).
* time marching: Carpenter-Kennedy LSRK(5,4) in 2N storage; the paper uses
  SDIRK but states (Sec. IV) that explicit RK of any order applies.
"""
import numpy as np

from . import mesh as _mesh
from . import ops as _ops
from . import velset as _velset

# Carpenter & Kennedy (1994) five-stage fourth-order 2N-storage coefficients.
LSRK_A = np.array([0.0,
                   -567301805773.0 / 1357537059087.0,
                   -2404267990393.0 / 2016746695238.0,
                   -3550918686646.0 / 2091501179385.0,
                   -1275806237668.0 / 842570457699.0])
LSRK_B = np.array([1432997174477.0 / 9575080441755.0,
                   5161836677717.0 / 13612068292357.0,
                   1720146321549.0 / 2090206949498.0,
                   3134564353537.0 / 4481467310338.0,
                   2277821191437.0 / 14882151754819.0])
LSRK_C = np.array([0.0,
                   1432997174477.0 / 9575080441755.0,
                   2526269341429.0 / 6820363962896.0,
                   2006345519317.0 / 3224310063776.0,
                   2802321613138.0 / 2924317926251.0])

SIDE_NORMAL = np.array([[0.0, -1.0], [1.0, 0.0], [0.0, 1.0], [-1.0, 0.0]])


def moments(f, ex, ey):
    """Nodal rho, u_x, u_y from f[..., Q] (Sec. II.A.2)."""
    rho = f.sum(axis=-1)
    jx = f @ ex
    jy = f @ ey
    return rho, jx / rho, jy / rho


def equilibrium(rho, ux, uy, ex, ey, w, eq_order=2):
    """Discrete Hermite equilibrium (eq. feq; third order from eq. Herm3a)."""
    rho = np.asarray(rho, dtype=np.float64)
    ux = np.asarray(ux, dtype=np.float64)[..., None]
    uy = np.asarray(uy, dtype=np.float64)[..., None]
    eu = ux * ex + uy * ey
    uu = ux * ux + uy * uy
    poly = 1.0 + eu + 0.5 * (eu * eu - uu)
    if eq_order == 3:
        poly = poly + eu * eu * eu / 6.0 - 0.5 * eu * uu
    return w * rho[..., None] * poly


def tau_from_kn(kn, L=1.0, cs=1.0, model="kn"):
    """Relaxation time from Kn (Sec. II.A.4).

    "kn": eq. KnTau, the mean free path lambda = sqrt(3) tau c_s and
          Kn = lambda / L, so tau = Kn L / (sqrt(3) c_s).
    "kim_pitsch": the mean free path of Kim and Pitsch from kinetic theory,
          lambda = tau c_s sqrt(pi / 2), which is sqrt(pi/6) times the one
          above (the paper's "additional factor of sqrt(pi/6)").
    "psi": eq. KnTau scaled by psi(Kn) = (2/pi) arctan(sqrt(2) Kn^(-3/4)).
    """
    if model == "kn":
        return kn * L / (np.sqrt(3.0) * cs)
    if model == "kim_pitsch":
        lam_per_tau = cs * np.sqrt(np.pi / 2.0)     # lambda / tau
        return kn * L / lam_per_tau
    if model == "psi":
        psi = 2.0 / np.pi * np.arctan(np.sqrt(2.0) * kn ** -0.75)
        return psi * tau_from_kn(kn, L, cs)
    raise ValueError(model)


class Problem:
    """One DG discrete-velocity BGK problem on a triangle mesh of a rectangle.

    The mesh is the structured Nx x Ny split-square mesh, or, when `mesh` =
    (vert_xy [nv, 2], tri [nt, 3]) is given, that conforming triangulation of
    [0, Lx] x [0, Ly] (counter-clockwise triangles; Nx, Ny, Lx, Ly are then
    ignored and the rectangle is read off the vertices).
    bc: 4 side kinds ('periodic' | 'diffuse' | 'eq') for sides
        0 (y=0), 1 (x=Lx), 2 (y=Ly), 3 (x=0); wall_u: 4 wall velocities.
    """

    def __init__(self, Nx, Ny, p, velset=("gh", 4), eq_order=2, kn=1.0, L=1.0,
                 beta=1.0, bc=("diffuse", "periodic", "diffuse", "periodic"),
                 wall_u=((-0.1, 0.0), (0.0, 0.0), (0.1, 0.0), (0.0, 0.0)),
                 cfl=0.5, dt=None, collision=True, Lx=1.0, Ly=1.0,
                 nc_extent=4.0, nc_scale=1.0, mesh=None, tau_model="kn"):
        self.Nx, self.Ny, self.p = Nx, Ny, p
        kind, n = velset
        self.ex, self.ey, self.w = _velset.velocity_set(kind, n, nc_extent, nc_scale)
        self.Q = len(self.w)
        self.eq_order = eq_order
        self.tau = tau_from_kn(kn, L, model=tau_model)
        self.collision = collision
        self.ab = 2.0 * beta - 1.0
        self.bc = tuple(bc)
        self.wall_u = np.array(wall_u, dtype=np.float64)
        assert (bc[1] == "periodic") == (bc[3] == "periodic")
        assert (bc[0] == "periodic") == (bc[2] == "periodic")
        self.ops = _ops.RefOps(p)
        self.Np, self.Nfp = self.ops.Np, self.ops.Nfp
        if mesh is None:
            self.vx, self.vy = _mesh.structured_mesh(Nx, Ny, Lx, Ly)
        else:
            self.vx, self.vy = _mesh.element_vertices(*mesh)
            Lx, Ly = float(self.vx.max()), float(self.vy.max())
        self.K = self.vx.shape[0]
        self.geo = _ops.geometry(self.vx, self.vy)
        self.x, self.y = _ops.physical_nodes(self.ops, self.vx, self.vy)
        self.nbr_elem, self.nbr_face, self.side = _mesh.connectivity(
            self.vx, self.vy, Lx, Ly, bc[1] == "periodic", bc[0] == "periodic")
        self._face_maps(Lx, Ly)
        self._wall_states()
        rin = _mesh.inscribed_radius(self.vx, self.vy).min()
        emax = np.sqrt(self.ex ** 2 + self.ey ** 2).max()
        self.dt = dt if dt is not None else cfl * rin / (emax * (p + 1) ** 2)

    # -- connectivity of face nodes, by matching physical coordinates --------
    def _face_maps(self, Lx, Ly):
        K, Nfp, fm = self.K, self.Nfp, self.ops.fmask
        self.mapk = np.zeros((K, 3, Nfp), dtype=np.int64)   # neighbour element
        self.mapn = np.zeros((K, 3, Nfp), dtype=np.int64)   # neighbour node
        for k in range(K):
            for f in range(3):
                kn, fn = self.nbr_elem[k, f], self.nbr_face[k, f]
                if kn < 0:                      # wall: placeholder = own trace
                    self.mapk[k, f] = k
                    self.mapn[k, f] = fm[f]
                    continue
                if self.p == 0:                 # single centroid node, no matching
                    self.mapk[k, f] = kn
                    self.mapn[k, f] = 0
                    continue
                shx = shy = 0.0
                s = self.side[k, f]
                if s == 1:
                    shx = Lx
                elif s == 3:
                    shx = -Lx
                elif s == 0:
                    shy = -Ly
                elif s == 2:
                    shy = Ly
                xm, ym = self.x[k, fm[f]], self.y[k, fm[f]]
                xp, yp = self.x[kn, fm[fn]] + shx, self.y[kn, fm[fn]] + shy
                for a in range(Nfp):
                    d = np.hypot(xp - xm[a], yp - ym[a])
                    b = int(np.argmin(d))
                    assert d[b] < 1e-10 * max(Lx, Ly)
                    self.mapk[k, f, a] = kn
                    self.mapn[k, f, a] = fm[fn][b]
        self.is_wall = self.nbr_elem < 0

    def _wall_states(self):
        """Per side: f^eq(1, u_b) and the denominator of eq. FullBC."""
        self.feq_b = np.zeros((4, self.Q))
        self.den_b = np.ones(4)
        for sd in range(4):
            u = self.wall_u[sd]
            self.feq_b[sd] = equilibrium(1.0, u[0], u[1], self.ex, self.ey, self.w, self.eq_order)
            n = SIDE_NORMAL[sd]
            en = self.ex * n[0] + self.ey * n[1]
            self.den_b[sd] = np.sum(np.where(en < 0, -en, 0.0) * self.feq_b[sd])

    # -- the residual ---------------------------------------------------------
    def rhs(self, f, elems=None):
        """df/dt at the nodes of `elems` (default: all), shape [len(elems), Np, Q].

        `f` is the full state [K, Np, Q]; neighbours are read from it.
        """
        if elems is None:
            elems = np.arange(self.K)
        elems = np.asarray(elems, dtype=np.int64)
        ops, g, Nfp = self.ops, self.geo, self.Nfp
        ex, ey, w = self.ex, self.ey, self.w
        fe = f[elems]
        # volume term -(e . grad) f
        fr = np.einsum("nm,kmq->knq", ops.Dr, fe)
        fs = np.einsum("nm,kmq->knq", ops.Ds, fe)
        ar = ex[None, :] * g["rx"][elems, None] + ey[None, :] * g["ry"][elems, None]
        as_ = ex[None, :] * g["sx"][elems, None] + ey[None, :] * g["sy"][elems, None]
        out = -(ar[:, None, :] * fr + as_[:, None, :] * fs)
        # surface term: lift of Fscale * (F^- - F^*).n
        flux = np.zeros((len(elems), 3 * Nfp, self.Q))
        for fc in range(3):
            fm = fe[:, ops.fmask[fc], :]
            fp = f[self.mapk[elems, fc], self.mapn[elems, fc], :]
            nx = g["nx"][elems, fc][:, None]
            ny = g["ny"][elems, fc][:, None]
            en = ex[None, :] * nx + ey[None, :] * ny                 # [E, Q]
            wall = self.is_wall[elems, fc]
            if np.any(wall):
                for idx in np.nonzero(wall)[0]:
                    sd = self.side[elems[idx], fc]
                    e_n = en[idx]
                    if self.bc[sd] == "diffuse":
                        num = (np.where(e_n > 0, e_n, 0.0)[None, :] * fm[idx]).sum(axis=1)  # [Nfp]
                        rho_w = num / self.den_b[sd]
                        inc = rho_w[:, None] * self.feq_b[sd][None, :]
                    else:  # "eq": eq. UsedBC with rho_b = 1
                        inc = np.broadcast_to(self.feq_b[sd][None, :], fm[idx].shape)
                    fp[idx] = np.where(e_n[None, :] < 0, inc, fm[idx])
            c = 0.5 * (en - self.ab * np.abs(en)) * g["Fscale"][elems, fc][:, None]
            flux[:, fc * Nfp:(fc + 1) * Nfp, :] = c[:, None, :] * (fm - fp)
        out += np.einsum("nj,kjq->knq", ops.LIFT, flux)
        if self.collision:
            rho, ux, uy = moments(fe, ex, ey)
            feq = equilibrium(rho, ux, uy, ex, ey, w, self.eq_order)
            out -= (fe - feq) / self.tau
        return out

    # -- time marching ---------------------------------------------------------
    def lsrk_stage(self, s, f, res, elems=None):
        """One 2N-storage stage: res <- A_s res + dt L(f); f <- f + B_s res."""
        res = LSRK_A[s] * res + self.dt * self.rhs(f, elems)
        fe = f if elems is None else f[elems]
        return fe + LSRK_B[s] * res, res

    def lsrk_step(self, f, res=None):
        if res is None:
            res = np.zeros_like(f)
        for s in range(5):
            f, res = self.lsrk_stage(s, f, res)
        return f, res

    def run(self, f, nsteps):
        res = np.zeros_like(f)
        for _ in range(nsteps):
            f, res = self.lsrk_step(f, res)
        return f

    # -- initial states and diagnostics ---------------------------------------
    def equilibrium_state(self, rho0=1.0, ux0=0.0, uy0=0.0, amp=0.0, u=None):
        """f = f^eq(rho0, u0) (1 + amp * u), u in [-1, 1) of shape [K, Np, Q]."""
        feq = equilibrium(np.full((self.K, self.Np), rho0), np.full((self.K, self.Np), ux0),
                          np.full((self.K, self.Np), uy0), self.ex, self.ey, self.w, self.eq_order)
        if u is None:
            return feq
        return feq * (1.0 + amp * u)

    def nodal_moments(self, f):
        return moments(f, self.ex, self.ey)

    def mass(self, f):
        """sum_k J_k 1^T M rho_k in FP64."""
        rho = f.sum(axis=-1)
        colsum = self.ops.M.sum(axis=0)
        return float(np.sum(self.geo["J"][:, None] * colsum[None, :] * rho))

    def l2_error(self, nodal, exact_fn, nq=8):
        """sqrt(sum_k int_Dk (u^e - u^k)^2) for a nodal field [K, Np] (Sec. III.A)."""
        qr, qs, qw = _ops.triangle_quadrature(nq)
        B, _, _ = _ops._basis(self.p, qr, qs)
        Bn, _, _ = _ops._basis(self.p, self.ops.r, self.ops.s)
        Lq = B @ np.linalg.inv(Bn)                       # [nq, Np]
        vx, vy = self.vx, self.vy
        xq = (-0.5 * (qr + qs))[None, :] * vx[:, :1] + (0.5 * (1 + qr))[None, :] * vx[:, 1:2] \
            + (0.5 * (1 + qs))[None, :] * vx[:, 2:3]
        yq = (-0.5 * (qr + qs))[None, :] * vy[:, :1] + (0.5 * (1 + qr))[None, :] * vy[:, 1:2] \
            + (0.5 * (1 + qs))[None, :] * vy[:, 2:3]
        uq = nodal @ Lq.T
        err = (exact_fn(xq, yq) - uq) ** 2
        return float(np.sqrt(np.sum(self.geo["J"][:, None] * qw[None, :] * err)))


def steady_state(problem, f0, pseudo_dt=1e3, tol=1e-13, max_iter=30):
    """Steady state by backward-Euler pseudo-time stepping with Newton.

    Backward Euler is the paper's own integrator for its steady cavity runs
    (Sec. II.B.3).  Each step solves (I/pdt - J) df = R(f) with a dense
    finite-difference Jacobian J = dR/df taken once at f0; it conserves mass
    exactly, which removes the mass null mode of R.  Small problems only.
    """
    shape = f0.shape
    n = f0.size
    f = f0.copy().ravel()

    def R(v):
        return problem.rhs(v.reshape(shape)).ravel()

    r0 = R(f)
    J = np.empty((n, n))
    h = 1e-7 * max(1.0, np.abs(f).max())
    for j in range(n):
        v = f.copy()
        v[j] += h
        J[:, j] = (R(v) - r0) / h
    from scipy.linalg import lu_factor, lu_solve
    lu = lu_factor(np.eye(n) / pseudo_dt - J)
    for _ in range(max_iter):
        r = R(f)
        if np.abs(r).max() < tol:
            break
        f = f + lu_solve(lu, r)
    return f.reshape(shape), float(np.abs(R(f)).max())
