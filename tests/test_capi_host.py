"""CPU tests of the C ABI library: it loads, exports every declared symbol, and
its host-side set-up (velocity sets, operators, mesh, time step) agrees with
the independently built oracle.  No GPU call is made here."""
import os
import re

import numpy as np
import pytest

from oracle import dg, ops, velset

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
fb = pytest.importorskip("paper_2012_13487_gb300.fedbm")


def _lib_or_skip():
    try:
        return fb.lib()
    except RuntimeError as e:
        pytest.skip(str(e))


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(fedbm_\w+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    L = _lib_or_skip()
    names = declared_symbols()
    assert len(names) >= 15
    for n in sorted(names):
        assert hasattr(L, n), n
    # and the binding wraps exactly these
    assert names == set(fb.SIGNATURES)


@pytest.mark.parametrize("kind,n,sq", [("gh", 4, 0), ("gh", 3, 0), ("gh", 18, 0), ("gh", 33, 0),
                                       ("nc", 16, 0), ("nc", 32, 0), ("nc", 33, 1)])
def test_velocity_sets_match_oracle(kind, n, sq):
    _lib_or_skip()
    d = fb.velset_desc(fb.VELSET_GH if kind == "gh" else fb.VELSET_NC, n, nc_sqrt2=sq)
    ex, ey, w = fb.fedbm_velset(d)
    oex, oey, ow = velset.velocity_set(kind, n, 4.0, np.sqrt(2.0) if sq else 1.0)
    np.testing.assert_allclose(ex, oex, atol=1e-13)
    np.testing.assert_allclose(ey, oey, atol=1e-13)
    np.testing.assert_allclose(w, ow, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("p", range(0, 7))
def test_reference_operators_match_oracle(p):
    _lib_or_skip()
    o = fb.fedbm_ref_operators(p)
    r = ops.RefOps(p)
    for k in ("r", "s", "Dr", "Ds", "LIFT", "M"):
        np.testing.assert_allclose(o[k], getattr(r, k), atol=1e-12 * max(1.0, np.abs(getattr(r, k)).max()))
    assert (o["fmask"] == r.fmask).all()


@pytest.mark.parametrize("nx,ny,p,bc", [(3, 2, 2, ("diffuse", "periodic", "diffuse", "periodic")),
                                        (1, 4, 3, ("diffuse", "periodic", "diffuse", "periodic")),
                                        (2, 3, 1, ("periodic",) * 4), (3, 3, 4, ("diffuse",) * 4),
                                        (4, 2, 0, ("eq", "periodic", "eq", "periodic"))])
def test_mesh_connectivity_nodes_and_dt_match_oracle(nx, ny, p, bc):
    _lib_or_skip()
    pr = dg.Problem(nx, ny, p, bc=bc)
    code = {"diffuse": 1, "periodic": 0, "eq": 2}
    m = fb.mesh_desc(nx, ny, p, bc=tuple(code[b] for b in bc))
    nbr = fb.fedbm_mesh_connectivity(m)
    fm = pr.ops.fmask
    for k in range(pr.K):
        for f in range(3):
            c = int(nbr[k, f])
            if c < 0:
                assert pr.nbr_elem[k, f] < 0 and -c - 1 == pr.side[k, f]
                continue
            kn, fn, rv = c >> 3, (c >> 1) & 3, c & 1
            assert kn == pr.nbr_elem[k, f] and fn == pr.nbr_face[k, f]
            if p > 0:
                for a in range(p + 1):
                    assert pr.mapn[k, f, a] == fm[fn][p - a if rv else a]
    x, y, dt = fb.fedbm_mesh_nodes(m, fb.velset_desc(), fb.params(cfl=0.5))
    np.testing.assert_allclose(x, pr.x, atol=1e-15)
    np.testing.assert_allclose(y, pr.y, atol=1e-15)
    assert dt == pytest.approx(pr.dt, rel=1e-14)


def test_invalid_descriptors_are_rejected():
    _lib_or_skip()
    with pytest.raises(fb.FedbmError) as e:
        fb.fedbm_velset(fb.velset_desc(fb.VELSET_GH, 0))
    assert e.value.code == fb.FEDBM_EINVAL
    with pytest.raises(fb.FedbmError):
        fb.fedbm_velset(fb.velset_desc(fb.VELSET_GH, 4, eq_order=5))
    with pytest.raises(fb.FedbmError):
        fb.fedbm_ref_operators(7)
    # one periodic side without its partner
    with pytest.raises(fb.FedbmError):
        fb.fedbm_mesh_connectivity(fb.mesh_desc(2, 2, 1, bc=(1, 0, 1, 1)))
    # a wall moving through itself
    with pytest.raises(fb.FedbmError):
        fb.fedbm_mesh_connectivity(fb.mesh_desc(2, 2, 1, bc=(1, 1, 1, 1), wall_u=((0, 0.1), (0, 0), (0, 0), (0, 0))))
