"""Walls on the fastest axis: a duct (the bumped, stretched channel of the
parity tests with a second pair of walls across its spanwise axis, which is
the fastest axis in memory, spanwise spacing uniform).

With the wall-link reading that takes Theta on wall-crossing links from the
extrapolated ghost nodes (wall_links = 1), the ghosts continue the uniform
spanwise spacing, so every cell of a row has the same geometry and the step
runs in plane mode. Along a row the first and last cells are wall cells and
the others are not: the step kernel takes its general neighbour addressing
(wall tests, reflected links) in the first and its wall-free addressing in
the others, and 16-bit storage relative to the column's rest state masks the
column differences of the links that a fastest-axis wall sends back. With
the other reading (wall_links = 0, Theta zero on wall-crossing links) the end
cells' link coefficients differ from the rest of the row: plane mode, and
with it the rest reference, is refused, and every cell streams its own record.

Every form is held to the FP64 oracle: FP64 at 1e-12 after 50 steps, FP32 at
2e-5 after 200 steps, 16-bit storage at the bounds of its rounding (those of
test_gpu_storage16). Even and odd row lengths take the two ways of finding a
16-bit value's half.
"""
import numpy as np
import pytest

from oracle import OracleSim
from paper_2401_17183_gb300 import workloads as W

from .helpers import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    from paper_2401_17183_gb300 import build as B
    B.build()
    from paper_2401_17183_gb300 import vlb
    vlb.load()
    return vlb


def duct_mesh(n0, n1, n2, wall_links):
    mesh = dict(W.channel_mesh(n0, n1, n2, stretch=0.7, bump=0.05, wall_links=wall_links))
    mesh["bc"] = (W.PERIODIC, W.WALL, W.WALL)
    shift = mesh["shift"].copy()
    shift[2] = 0.0
    mesh["shift"] = shift
    return mesh


def _oracle_run(mesh):
    prm = W.params(0.6, body_force=(1e-5, 0, 0))
    rho, u = W.noise_fields(mesh, amp=0.01, seed=2)
    o = OracleSim(mesh, prm)
    o.init(rho, u)
    m0 = o.moments()
    o.step(50)
    m50 = o.moments()
    o.step(150)
    return mesh, prm, rho, u, m0, m50, o.moments()


@pytest.fixture(scope="module", params=[(16, 12, 8), (15, 12, 7)], ids=["even-rows", "odd-rows"])
def duct(request):
    return _oracle_run(duct_mesh(*request.param, wall_links=1))


@pytest.fixture(scope="module")
def duct_records():
    return _oracle_run(duct_mesh(16, 12, 8, wall_links=0))


def _cmp(gm, om, tol_rho, tol_u):
    assert rel_err(gm["rho"], om["rho"], 1.0) < tol_rho
    su = np.abs(om["u"]).max()
    assert rel_err(gm["u"], om["u"], su) < tol_u
    assert rel_err(gm["u_tilde"], om["u_tilde"], su) < tol_u


def test_duct_fp64_both_coefficient_modes(V, duct):
    mesh, prm, rho, u, _, m50, _ = duct
    for mode in (V.VLB_COEF_FULL, V.VLB_COEF_PLANE):
        g = V.Sim(V.Mesh(mesh), prm, rho, u, precision=V.VLB_F64, coef_mode=mode)
        assert g.layout()["plane"] == (mode == V.VLB_COEF_PLANE)
        g.step(50)
        gm = g.moments()
        _cmp(gm, m50, 1e-12, 1e-12)
        assert abs(gm["mass"] - m50["mass"]) <= 1e-12 * m50["mass"]


def test_duct_fp32(V, duct):
    mesh, prm, rho, u, _, _, m200 = duct
    g = V.Sim(V.Mesh(mesh), prm, rho, u, precision=V.VLB_F32)
    assert g.layout()["plane"]
    g.step(200)
    _cmp(g.moments(), m200, 2e-5, 2e-5)


# (precision, reference, max error of u (to max|u|), of rho, of the mass drift
# over 200 steps): the bounds of the 16-bit channel test
CASES = [("F16", "REST", 1e-3, 5e-4, 2e-5), ("F16", "UNIFORM", 2e-3, 1e-3, 2e-5),
         ("BF16", "REST", 1e-2, 5e-3, 2e-4)]


@pytest.mark.parametrize("case", CASES, ids=["%s-%s" % c[:2] for c in CASES])
def test_duct_16bit(V, duct, case):
    mesh, prm, rho, u, _, _, m200 = duct
    prec, ref, tol_u, tol_rho, tol_mass = case
    g = V.Sim(V.Mesh(mesh), prm, rho, u, precision=getattr(V, "VLB_" + prec),
              reference=getattr(V, "VLB_REF_" + ref))
    assert g.layout()["plane"]
    mi = g.moments(fields=False)["mass"]
    g.step(200)
    gm = g.moments()
    _cmp(gm, m200, tol_rho, tol_u)
    assert abs(gm["mass"] - mi) <= tol_mass * mi


def test_duct_without_ghost_links_streams_records(V, duct_records):
    mesh, prm, rho, u, _, m50, m200 = duct_records
    gm = V.Mesh(mesh)
    for kw in ({"precision": V.VLB_F64, "coef_mode": V.VLB_COEF_PLANE},
               {"precision": V.VLB_F16, "reference": V.VLB_REF_REST}):
        with pytest.raises(V.VlbError) as e:
            V.Sim(gm, prm, rho, u, **kw)
        assert e.value.code == "EINVAL"
    g = V.Sim(gm, prm, rho, u, precision=V.VLB_F64)
    assert not g.layout()["plane"]
    g.step(50)
    _cmp(g.moments(), m50, 1e-12, 1e-12)
    g = V.Sim(gm, prm, rho, u, precision=V.VLB_F32)
    g.step(200)
    _cmp(g.moments(), m200, 2e-5, 2e-5)
