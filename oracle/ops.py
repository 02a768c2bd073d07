"""Nodal DG operators on the reference triangle (Sec. II.B.1).  Test
infrastructure only.

Reference triangle: vertices (-1,-1), (1,-1), (-1,1) in (r, s).  The nodal
set is the warp & blend construction of Warburton (2006) with alpha = 0
(the paper does not name its node set; this is the reading used by both
sides).  Nodes are numbered row by row: for row i = 0..p (the s direction),
column j = 0..p-i (the r direction).

Construction (independent of the CUDA library's own): the interpolating
basis is expanded in unnormalised Proriol-Koornwinder-Dubiner polynomials
evaluated with SciPy's Jacobi routine; Dr = Vr V^-1, Ds = Vs V^-1; the mass
matrix is integrated with a collapsed-coordinate Gauss rule and each face
mass matrix with a 1-D Gauss-Legendre rule along the face; LIFT = M^-1 E.

Faces (counter-clockwise vertex order v0 -> v1 -> v2):
  face 0: s = -1 (v0 -> v1), parameter t = r,
  face 1: r + s = 0 (v1 -> v2), parameter t = s,
  face 2: r = -1 (v2 -> v0), parameter t = s,
face nodes listed in increasing t.
"""
import numpy as np
from numpy.polynomial import legendre as npleg
from scipy.special import eval_jacobi


def gll_points(p):
    """p+1 Gauss-Lobatto-Legendre points on [-1, 1]: +-1 and the roots of P_p'."""
    if p == 0:
        return np.array([0.0])
    if p == 1:
        return np.array([-1.0, 1.0])
    dP = npleg.Legendre.basis(p).deriv()
    inner = np.sort(np.real(dP.roots()))
    return np.concatenate(([-1.0], inner, [1.0]))


def _lagrange_eval(xnodes, j, x):
    """j-th Lagrange polynomial on xnodes evaluated at x."""
    out = np.ones_like(x)
    for m, xm in enumerate(xnodes):
        if m != j:
            out = out * (x - xm) / (xnodes[j] - xm)
    return out


def _warp(p, rout):
    """1-D warp: GLL minus equispaced, interpolated on equispaced points and
    divided by (1 - r^2) away from the end points (the blend denominator)."""
    req = np.linspace(-1.0, 1.0, p + 1)
    gll = gll_points(p)
    warp = np.zeros_like(rout)
    for j in range(p + 1):
        warp += (gll[j] - req[j]) * _lagrange_eval(req, j, rout)
    inside = np.abs(rout) < 1.0 - 1e-10
    warp = np.where(inside, warp / np.where(inside, 1.0 - rout * rout, 1.0), 0.0)
    return warp


def nodes(p):
    """Warp & blend nodes (alpha = 0) on the reference triangle: (r, s), [Np]."""
    if p == 0:
        return np.array([-1.0 / 3.0]), np.array([-1.0 / 3.0])
    L1, L3 = [], []
    for i in range(p + 1):          # row (s direction)
        for j in range(p + 1 - i):  # column (r direction)
            L1.append(i / p)
            L3.append(j / p)
    L1 = np.array(L1)
    L3 = np.array(L3)
    L2 = 1.0 - L1 - L3
    # equilateral triangle (-1,-1/sqrt3), (1,-1/sqrt3), (0, 2/sqrt3)
    X = -L2 + L3
    Y = (-L2 - L3 + 2.0 * L1) / np.sqrt(3.0)
    w1 = 4.0 * L2 * L3 * _warp(p, L3 - L2)
    w2 = 4.0 * L1 * L3 * _warp(p, L1 - L3)
    w3 = 4.0 * L1 * L2 * _warp(p, L2 - L1)
    X = X + w1 + np.cos(2 * np.pi / 3) * w2 + np.cos(4 * np.pi / 3) * w3
    Y = Y + np.sin(2 * np.pi / 3) * w2 + np.sin(4 * np.pi / 3) * w3
    # equilateral -> reference (barycentric coordinates are preserved)
    b1 = (np.sqrt(3.0) * Y + 1.0) / 3.0
    b2 = (-3.0 * X - np.sqrt(3.0) * Y + 2.0) / 6.0
    b3 = (3.0 * X - np.sqrt(3.0) * Y + 2.0) / 6.0
    r = -b2 + b3 - b1
    s = -b2 - b3 + b1
    return r, s


def face_masks(p):
    """Node indices on faces 0, 1, 2, each ordered by increasing t: [3, p+1]."""
    rows = []
    start = 0
    for i in range(p + 1):
        rows.append(list(range(start, start + p + 1 - i)))
        start += p + 1 - i
    f0 = rows[0]
    f1 = [rows[i][-1] for i in range(p + 1)]
    f2 = [rows[i][0] for i in range(p + 1)]
    return np.array([f0, f1, f2], dtype=np.int64)


def _basis(p, r, s):
    """Proriol-Koornwinder-Dubiner polynomials and their r, s derivatives.

    psi_ij = P_i(a) P_j^(2i+1,0)(b) (1-b)^i with collapsed coordinates
    a = 2(1+r)/(1-s) - 1, b = s (a = -1 at the vertex s = 1), evaluated with
    SciPy's (unnormalised) Jacobi polynomials; derivatives by the chain rule
    with dP_n^(al,be)/dx = (n+al+be+1)/2 P_(n-1)^(al+1,be+1).  Only the span
    matters: every operator below is formed through V^-1.
    """
    r = np.asarray(r, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    top = np.abs(1.0 - s) < 1e-14
    a = np.where(top, -1.0, 2.0 * (1.0 + r) / np.where(top, 1.0, 1.0 - s) - 1.0)
    b = s
    om = 1.0 - b

    def jac(n, al, be, x):
        return eval_jacobi(n, al, be, x) if n >= 0 else np.zeros_like(x)

    def djac(n, al, be, x):
        return 0.5 * (n + al + be + 1) * jac(n - 1, al + 1, be + 1, x) if n > 0 else np.zeros_like(x)

    cols, dcr, dcs = [], [], []
    for i in range(p + 1):
        for j in range(p + 1 - i):
            A, dA = jac(i, 0, 0, a), djac(i, 0, 0, a)
            B, dB = jac(j, 2 * i + 1, 0, b), djac(j, 2 * i + 1, 0, b)
            cols.append(A * B * om ** i)
            if i == 0:
                dcr.append(np.zeros_like(r))
                dcs.append(A * dB)
            else:
                dcr.append(2.0 * dA * B * om ** (i - 1))
                dcs.append(dA * (1.0 + a) * B * om ** (i - 1) + A * dB * om ** i
                           - i * A * B * om ** (i - 1))
    return np.array(cols).T, np.array(dcr).T, np.array(dcs).T


def triangle_quadrature(nq):
    """Collapsed-coordinate Gauss rule on the reference triangle (area 2)."""
    g, gw = npleg.leggauss(nq)
    A, B = np.meshgrid(g, g, indexing="ij")
    WA, WB = np.meshgrid(gw, gw, indexing="ij")
    r = 0.5 * (1.0 + A) * (1.0 - B) - 1.0
    s = B
    w = WA * WB * 0.5 * (1.0 - B)
    return r.ravel(), s.ravel(), w.ravel()


class RefOps:
    """Reference-element operators for order p.

    Dr, Ds  : [Np, Np] nodal derivative matrices (d/dr, d/ds of the
              interpolant, evaluated at the nodes).
    M       : [Np, Np] mass matrix int l_i l_j.
    Emat    : [Np, 3*Nfp] face mass matrices int_face l_i l^face_a dt.
    LIFT    : M^-1 Emat.
    fmask   : [3, Nfp] face nodes.
    """

    def __init__(self, p):
        self.p = p
        self.Np = (p + 1) * (p + 2) // 2
        self.Nfp = p + 1
        self.r, self.s = nodes(p)
        self.fmask = face_masks(p)
        V, Vr, Vs = _basis(p, self.r, self.s)
        Vinv = np.linalg.inv(V)
        self.Dr = Vr @ Vinv
        self.Ds = Vs @ Vinv
        # mass matrix by quadrature of the Lagrange basis
        qr, qs, qw = triangle_quadrature(p + 3)
        Bq, _, _ = _basis(p, qr, qs)
        Lq = Bq @ Vinv                       # [nq, Np] Lagrange basis at quad points
        self.M = Lq.T @ (qw[:, None] * Lq)
        # face mass matrices
        Nfp = self.Nfp
        g, gw = npleg.leggauss(p + 3)
        E = np.zeros((self.Np, 3 * Nfp))
        for f in range(3):
            if f == 0:
                rr, ss = g, -np.ones_like(g)
                tnodes = self.r[self.fmask[0]]
            elif f == 1:
                rr, ss = -g, g
                tnodes = self.s[self.fmask[1]]
            else:
                rr, ss = -np.ones_like(g), g
                tnodes = self.s[self.fmask[2]]
            Bf, _, _ = _basis(p, rr, ss)
            Lf = Bf @ Vinv                   # triangle Lagrange basis on the face
            for a in range(Nfp):
                la = _lagrange_eval(tnodes, a, g) if Nfp > 1 else np.ones_like(g)
                E[:, f * Nfp + a] = (Lf * (gw * la)[:, None]).sum(axis=0)
        self.Emat = E
        self.LIFT = np.linalg.solve(self.M, E)


def geometry(vx, vy):
    """Affine geometric factors of every element.

    Returns a dict with rx, sx, ry, sy, J  ([K]) and nx, ny, sJ, Fscale
    ([K, 3]); faces as in the module docstring, normals outward.
    """
    xr = 0.5 * (vx[:, 1] - vx[:, 0])
    xs = 0.5 * (vx[:, 2] - vx[:, 0])
    yr = 0.5 * (vy[:, 1] - vy[:, 0])
    ys = 0.5 * (vy[:, 2] - vy[:, 0])
    J = xr * ys - xs * yr
    geo = dict(rx=ys / J, sx=-yr / J, ry=-xs / J, sy=xr / J, J=J)
    nx = np.zeros((vx.shape[0], 3))
    ny = np.zeros_like(nx)
    sJ = np.zeros_like(nx)
    for f in range(3):
        a, b = f, (f + 1) % 3
        dx = vx[:, b] - vx[:, a]
        dy = vy[:, b] - vy[:, a]
        length = np.hypot(dx, dy)
        nx[:, f] = dy / length
        ny[:, f] = -dx / length
        sJ[:, f] = 0.5 * length
    geo.update(nx=nx, ny=ny, sJ=sJ, Fscale=sJ / J[:, None])
    return geo


def physical_nodes(ops, vx, vy):
    """Physical coordinates x, y of every node, [K, Np]."""
    r, s = ops.r, ops.s
    x = (-0.5 * (r + s))[None, :] * vx[:, :1] + (0.5 * (1 + r))[None, :] * vx[:, 1:2] \
        + (0.5 * (1 + s))[None, :] * vx[:, 2:3]
    y = (-0.5 * (r + s))[None, :] * vy[:, :1] + (0.5 * (1 + r))[None, :] * vy[:, 1:2] \
        + (0.5 * (1 + s))[None, :] * vy[:, 2:3]
    return x, y
