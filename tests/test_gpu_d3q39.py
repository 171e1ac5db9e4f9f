"""GPU parity of the 6th-order isotropic velocity set D3Q39 (FP64, periodic
meshes) against the FP64 CPU oracle on the same seeded inputs: the geometry
of every direction (speeds up to 3), the populations after one, two and three
steps (both A-A parities) and after 20, the moments, the conservation of
mass and of the momentum invariant M(t), and the cases the path rejects.
"""
import numpy as np
import pytest

from oracle import OracleSim
from oracle import lattice as olat
from paper_2401_17183_gb300 import workloads as W

from .helpers import oracle_state_in_lib_order, perm, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    from paper_2401_17183_gb300 import build as B
    B.build()
    from paper_2401_17183_gb300 import vlb
    vlb.load()
    return vlb


def _case():
    mesh = W.periodic_sine_mesh3d(8, 0.01, q=39)
    prm = W.params(0.8, body_force=(1e-5, 0.0, 2e-6))
    rho, u = W.noise_fields(mesh, amp=0.02, seed=7, rho_amp=0.01)
    return mesh, prm, rho, u


def test_d3q39_lattice_and_geometry(V):
    mesh, prm, rho, u = _case()
    cl, wl = V.lattice(39)
    co, wo, _ = olat(39)
    p = perm(cl, co)
    assert np.array_equal(co[p], cl) and np.allclose(wo[p], wl, rtol=0, atol=1e-17)
    gm = V.Mesh(mesh).geometry()
    om = OracleSim(mesh, prm).geometry()
    assert rel_err(gm["J"], om["J"]) < 1e-13
    Ko = np.einsum("naij,aj->nai", om["theta"], co.astype(float))[:, p, :]
    assert np.abs(gm["K"] - Ko).max() <= 1e-13 * max(np.abs(Ko).max(), 1e-3)


def test_d3q39_steps_against_oracle(V):
    mesh, prm, rho, u = _case()
    g = V.Sim(V.Mesh(mesh), prm, rho, u, precision=V.VLB_F64)
    o = OracleSim(mesh, prm)
    o.init(rho, u)
    co, _, _ = olat(39)
    cl, _ = V.lattice(39)
    m0 = g.moments()
    done = 0
    for s in (1, 2, 3, 20):
        g.step(s - done)
        o.step(s - done)
        done = s
        exp = oracle_state_in_lib_order(o.get_state(), co, cl)
        assert rel_err(g.get_state(), exp) < (1e-13 if s <= 3 else 1e-12), s
    gm, om = g.moments(), o.moments()
    su = np.abs(om["u"]).max()
    assert rel_err(gm["rho"], om["rho"], 1.0) < 1e-12
    assert rel_err(gm["u"], om["u"], su) < 1e-12
    assert rel_err(gm["u_tilde"], om["u_tilde"], su) < 1e-12
    assert abs(gm["mass"] - m0["mass"]) <= 1e-13 * m0["mass"]
    assert abs(gm["mass"] - om["mass"]) <= 1e-13 * om["mass"]
    assert np.abs(gm["M"] - om["M"]).max() <= 1e-12 * np.abs(om["M"]).max() + 1e-14


def test_d3q39_state_roundtrip(V):
    mesh, prm, rho, u = _case()
    g = V.Sim(V.Mesh(mesh), prm, rho, u, precision=V.VLB_F64)
    g.step(3)
    N = g.get_state()
    g.set_state(N)          # back at time 0 with the same arrived populations
    assert np.array_equal(g.get_state(), N)
    h = V.Sim(V.Mesh(mesh), prm, rho, u, precision=V.VLB_F64)
    h.step(3)
    g.step(2)
    h.step(2)
    assert rel_err(g.get_state(), h.get_state()) < 1e-14


@pytest.mark.parametrize("case", ["f32", "wall", "plane", "noalloc"])
def test_d3q39_rejections(V, case):
    torch = pytest.importorskip("torch")
    mesh, prm, rho, u = _case()
    with pytest.raises(V.VlbError) as e:
        if case == "f32":
            V.Sim(V.Mesh(mesh), prm, rho, u, precision=V.VLB_F32)
        elif case == "wall":
            m = W.channel_mesh(6, 6, 6, stretch=0.7, bump=0.0)
            m["q"] = 39
            V.Mesh(m)
        elif case == "plane":
            V.Sim(V.Mesh(mesh), prm, rho, u, precision=V.VLB_F64, coef_mode=V.VLB_COEF_PLANE)
        else:
            g = V.Sim(V.Mesh(mesh), prm, rho, u, precision=V.VLB_F64)
            d = torch.zeros(7, dtype=torch.float64, device="cuda")
            g.totals_noalloc(d.data_ptr())
    assert e.value.code == "EINVAL"
