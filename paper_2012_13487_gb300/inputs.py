"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

Holds no arithmetic of the method: only a counter-based uniform generator.
SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) is applied to ``seed XOR index``; the top 53 bits
of the mixed word give a uniform double in [0, 1), mapped to [-1, 1).  The
index of a state entry is its canonical position (k*Np + j)*Q + i, so the
draw does not depend on any internal layout.  The CUDA library implements
the same published generator in its own code for ``fedbm_set_equilibrium``.
"""
import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x):
    """One SplitMix64 output for each uint64 state value in x."""
    z = np.asarray(x, dtype=np.uint64) + _GAMMA
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform_pm1(seed, n, start=0):
    """n doubles in [-1, 1) for canonical indices start .. start+n-1."""
    idx = np.arange(start, start + n, dtype=np.uint64)
    z = splitmix64(np.uint64(seed) ^ idx)
    u01 = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u01 - 1.0


def perturbation(seed, K, Np, Q):
    """Uniform [-1, 1) field of shape [K, Np, Q] (canonical layout)."""
    with np.errstate(over="ignore"):
        return uniform_pm1(seed, K * Np * Q).reshape(K, Np, Q)


def uniform01(seed, n, start=0):
    """n doubles in [0, 1) from SplitMix64(seed XOR index)."""
    idx = np.arange(start, start + n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = splitmix64(np.uint64(seed) ^ idx)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def batch_cases(seed=201213487, n=256):
    """Seeded mix of n independent cases: the first half Couette, the rest
    lid-driven cavity; Kn log-uniform in [0.5, 8]; wall or lid speed uniform
    in [0.05, 0.2] sqrt(RT); N x N x 2 triangles with N uniform in 16..64;
    degree uniform in 2..5; velocity set GH D2Q16 or NC 16 x 16 with
    probability 1/2 each.  Returns a list of dicts (draws only)."""
    u = uniform01(seed, 5 * n).reshape(n, 5)
    out = []
    for c in range(n):
        out.append(dict(
            kind="couette" if c < n // 2 else "cavity",
            kn=float(np.exp(np.log(0.5) + u[c, 0] * (np.log(8.0) - np.log(0.5)))),
            speed=float(0.05 + 0.15 * u[c, 1]),
            N=int(16 + min(48, int(u[c, 2] * 49))),
            p=int(2 + min(3, int(u[c, 3] * 4))),
            vel=("gh", 4) if u[c, 4] < 0.5 else ("nc", 16),
        ))
    return out


def unstructured_square(nx, ny, seed, jitter=0.2, shuffle=True, lx=1.0, ly=1.0):
    """A seeded conforming triangulation of [0, lx] x [0, ly] with irregular
    connectivity: an (nx+1) x (ny+1) vertex grid whose interior vertices are
    moved by up to `jitter` cell widths in each direction (boundary vertices
    slide along their side, corners stay), every cell split along a randomly
    chosen diagonal, each triangle's vertex list rotated by a random amount
    (it stays counter-clockwise) and, with `shuffle`, the triangles put in a
    random order.  Opposite sides keep the same vertex positions along the
    side, so they can be paired periodically.  Returns (vert_xy [nv, 2],
    tri [nt, 3] int32), nt = 2 nx ny.  Draws only; no arithmetic of the method."""
    nv = (nx + 1) * (ny + 1)
    u = uniform01(seed, 2 * nv + 2 * nx * ny + 2 * nx * ny).reshape(-1)
    jx = (2.0 * u[:nv] - 1.0) * jitter
    jy = (2.0 * u[nv:2 * nv] - 1.0) * jitter
    hx, hy = lx / nx, ly / ny
    vert = np.zeros((nv, 2))
    for iy in range(ny + 1):
        for ix in range(nx + 1):
            v = iy * (nx + 1) + ix
            x, y = ix * hx, iy * hy
            inner_x = 0 < ix < nx
            inner_y = 0 < iy < ny
            # side vertices move along their side only; a top (right) side
            # vertex takes the draw of the bottom (left) one below (beside) it,
            # so that opposite sides stay paired
            if inner_x:
                x += jx[v if inner_y else ix] * hx
            if inner_y:
                y += jy[v if inner_x else iy * (nx + 1)] * hy
            vert[v] = (x, y)
    diag = u[2 * nv:2 * nv + nx * ny] < 0.5
    rot = (u[2 * nv + nx * ny:2 * nv + 3 * nx * ny] * 3).astype(np.int64).clip(0, 2)
    tris = []
    for iy in range(ny):
        for ix in range(nx):
            a = iy * (nx + 1) + ix
            b, c, d = a + 1, a + nx + 2, a + nx + 1           # counter-clockwise corners
            cell = iy * nx + ix
            pair = ((a, b, c), (a, c, d)) if diag[cell] else ((a, b, d), (b, c, d))
            tris.extend(pair)
    tri = np.array(tris, dtype=np.int64)
    r = rot[:len(tri)]
    tri = np.stack([tri[np.arange(len(tri)), (r + j) % 3] for j in range(3)], axis=1)
    if shuffle:
        order = np.argsort(uniform01(seed ^ 0x5DEECE66D, len(tri)), kind="stable")
        tri = tri[order]
    X = vert[tri]
    area2 = (X[:, 1, 0] - X[:, 0, 0]) * (X[:, 2, 1] - X[:, 0, 1]) - (X[:, 2, 0] - X[:, 0, 0]) * (X[:, 1, 1] - X[:, 0, 1])
    if area2.min() < 0.1 * hx * hy:
        raise ValueError("jitter too large: a triangle lost most of its area")
    return vert, tri.astype(np.int32)
