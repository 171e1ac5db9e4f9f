"""16-bit population storage (IEEE half, bfloat16) with FP32 arithmetic.

Storage rounds every population to 11 (half) or 8 (bfloat16) significant bits
of its deviation from the storage reference, so these runs are compared with
the FP64 oracle (or the FP64 GPU path, which equals it to 1e-12) at
tolerances set by that rounding, not by the arithmetic:

  - the D3Q19 channel of the FP32 parity test (16 x 12 x 8, tau = 0.6, 200
    steps) for both storage types and both references;
  - on a 32^3 channel the local rest-state reference (only the flow is
    stored) is several times more accurate than the uniform one;
  - a stretched D2Q9 channel in plane mode;
  - state scatter/gather, the allocation-free totals and the error path.
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


# An even fastest axis lets the kernel tell a 16-bit value's half from the
# cell parity; an odd one takes the path that records the half per value.
@pytest.fixture(scope="module", params=[(16, 12, 8), (15, 12, 7)], ids=["even-rows", "odd-rows"])
def channel(request):
    mesh = W.channel_mesh(*request.param, stretch=0.7, bump=0.05)
    prm = W.params(0.6, body_force=(1e-5, 0, 0))
    rho, u = W.noise_fields(mesh, amp=0.01, seed=2)
    o = OracleSim(mesh, prm)
    o.init(rho, u)
    m0 = o.moments()
    o.step(200)
    return mesh, prm, rho, u, m0, o.moments()


# (precision name, reference, max rel. error of u (to max|u|), of rho, of the mass drift over
# 200 steps). Rounding a population to 16 bits does not conserve mass; the
# drift of the total over the run, measured from the run's own (rounded)
# start, was at most 4.1e-6 (FP16) and 4.4e-5 (bfloat16) over the four cases
# and both row parities, so the bounds leave a factor of about five.
CASES = [("F16", "REST", 1e-3, 5e-4, 2e-5), ("F16", "UNIFORM", 2e-3, 1e-3, 2e-5),
         ("BF16", "REST", 1e-2, 5e-3, 2e-4), ("BF16", "UNIFORM", 1e-2, 5e-3, 2e-4)]


@pytest.mark.parametrize("case", CASES, ids=["%s-%s" % c[:2] for c in CASES])
def test_channel_16bit_against_oracle(V, channel, case):
    mesh, prm, rho, u, m0, m200 = channel
    prec, ref, tol_u, tol_rho, tol_mass = case
    g = V.Sim(V.Mesh(mesh), prm, rho, u, precision=getattr(V, "VLB_" + prec),
              reference=getattr(V, "VLB_REF_" + ref))
    assert g.layout()["plane"]
    # the initial state is already rounded to the storage type
    mi = g.moments(fields=False)["mass"]
    assert abs(mi - m0["mass"]) <= 50 * tol_mass * m0["mass"]
    g.step(200)
    gm = g.moments()
    su = np.abs(m200["u"]).max()
    assert rel_err(gm["u"], m200["u"], su) < tol_u
    assert rel_err(gm["rho"], m200["rho"], 1.0) < tol_rho
    # drift of the total mass over the run, from storage rounding alone
    assert abs(gm["mass"] - mi) <= tol_mass * mi


def test_rest_reference_beats_uniform_on_stretched_mesh(V):
    """On the stretched, bumped channel most of a population's deviation from
    a uniform reference is the cell-volume and metric variation; storing
    relative to the local rest state leaves only the flow to be rounded."""
    mesh = W.channel_mesh(32, 32, 32, stretch=0.7, bump=0.05)
    prm = W.params(0.8, body_force=(1e-5, 0, 0))
    rho, u = W.noise_fields(mesh, amp=0.01, seed=2)
    gm = V.Mesh(mesh)
    ref = V.Sim(gm, prm, rho, u, precision=V.VLB_F64)
    ref.step(300)
    mr = ref.moments()
    su = np.abs(mr["u"]).max()
    errs = {}
    for name in ("REST", "UNIFORM"):
        s = V.Sim(gm, prm, rho, u, precision=V.VLB_F16, reference=getattr(V, "VLB_REF_" + name))
        s.step(300)
        errs[name] = rel_err(s.moments()["u"], mr["u"], su)
    assert errs["REST"] < 1e-3
    assert errs["REST"] * 3 < errs["UNIFORM"], errs


def test_channel2d_d2q9_16bit(V):
    """D2Q9 in plane mode: a stretched 2D channel driven by a body force along
    its periodic axis, against the FP64 GPU path."""
    mesh = W.channel2d_mesh(32, 16, stretch=0.7)
    prm = W.params(0.8, body_force=(0.0, 1e-5, 0.0))
    rho, u = W.noise_fields(mesh, amp=0.01, seed=3)
    gm = V.Mesh(mesh)
    ref = V.Sim(gm, prm, rho, u, precision=V.VLB_F64)
    ref.step(500)
    mr = ref.moments()
    su = np.abs(mr["u"]).max()
    for prec, tol in (("F16", 2e-3), ("BF16", 2e-2)):
        s = V.Sim(gm, prm, rho, u, precision=getattr(V, "VLB_" + prec), reference=V.VLB_REF_REST)
        assert s.layout()["plane"]
        s.step(500)
        sm = s.moments()
        assert rel_err(sm["u"], mr["u"], su) < tol, prec
        assert rel_err(sm["u_tilde"], mr["u_tilde"], su) < tol, prec


@pytest.mark.parametrize("prec", ["F16", "BF16"])
def test_state_roundtrip_16bit(V, prec):
    """Scatter then gather rounds each population once (relative to its
    storage reference); a second round trip changes nothing."""
    mesh = W.channel_mesh(16, 12, 8, stretch=0.7, bump=0.05)
    rho, u = W.noise_fields(mesh, amp=0.01, seed=4)
    s = V.Sim(V.Mesh(mesh), W.params(0.8), rho, u, precision=getattr(V, "VLB_" + prec),
              reference=V.VLB_REF_REST)
    s.step(3)
    N = s.get_state()
    s.set_state(N)
    N1 = s.get_state()
    s.set_state(N1)
    N2 = s.get_state()
    assert np.array_equal(N1, N2)
    bits = 11 if prec == "F16" else 8
    assert np.abs(N1 - N).max() <= 2.0 ** -bits * 0.25 * np.abs(N).max()


def test_totals_noalloc_16bit(V):
    torch = pytest.importorskip("torch")
    mesh = W.channel_mesh(24, 16, 12, stretch=0.7, bump=0.05)
    rho, u = W.noise_fields(mesh, amp=0.01, seed=2)
    s = V.Sim(V.Mesh(mesh), W.params(0.8, body_force=(1e-5, 0, 0)), rho, u,
              precision=V.VLB_F16, reference=V.VLB_REF_REST)
    s.step(5)
    out = torch.full((7,), float("nan"), dtype=torch.float64, device="cuda")
    s.totals_noalloc(out.data_ptr())
    s.sync()
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    m = s.moments(fields=False)
    exp = np.concatenate([[m["mass"]], m["P"], m["M"]])
    assert np.abs(got - exp).max() <= 1e-12 * exp[0]


def test_rest_reference_needs_plane_mode(V):
    mesh = W.channel_mesh(16, 12, 8, stretch=0.7, bump=0.05)
    rho, u = W.noise_fields(mesh, amp=0.01, seed=2)
    with pytest.raises(V.VlbError) as e:
        V.Sim(V.Mesh(mesh), W.params(0.8), rho, u, precision=V.VLB_F16,
              coef_mode=V.VLB_COEF_FULL, reference=V.VLB_REF_REST)
    assert e.value.code == "EINVAL"
    # the uniform reference works in either mode
    s = V.Sim(V.Mesh(mesh), W.params(0.8), rho, u, precision=V.VLB_F16, coef_mode=V.VLB_COEF_FULL)
    s.step(2)
    s.sync()
