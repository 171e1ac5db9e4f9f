"""vlb_totals_noalloc, the entry point for callers that cannot allocate device
memory (fixed memory budgets, pool allocators they do not own, latency-bound
loops): its totals must equal those of vlb_moments, call after call.

Kept in a file of its own that pytest collects last. Device memory for the
output comes from torch, as it would from such a caller's own pool.
"""
import numpy as np
import pytest

from paper_2401_17183_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2401_17183_gb300 import build as B
    B.build()
    from paper_2401_17183_gb300 import vlb
    vlb.load()
    return vlb


def _expected(m, dim):
    t = np.zeros(7)
    t[0] = m["mass"]
    t[1:1 + dim] = m["P"]
    t[4:4 + dim] = m["M"]
    return t


@pytest.mark.parametrize("case", ["channel_f32", "channel_f64", "wedge_f64"])
def test_totals_noalloc_matches_moments_on_consecutive_calls(case):
    torch = pytest.importorskip("torch")
    V = _lib()
    if case.startswith("channel"):
        mesh = W.channel_mesh(24, 16, 12, stretch=0.7, bump=0.05)
        prm = W.params(0.8, body_force=(1e-5, 0, 0))
        rho, u = W.noise_fields(mesh, amp=0.01, seed=2)
    else:
        mesh = W.polar_mesh(16, 3, 30.0, 36.0, dtheta=1.0 / 33)
        prm = W.params(0.9)
        rho, u = W.noise_fields(mesh, amp=0.01, seed=3)
    prec = V.VLB_F32 if case.endswith("f32") else V.VLB_F64
    sim = V.Sim(V.Mesh(mesh), prm, rho, u, precision=prec)
    out = torch.full((7,), float("nan"), dtype=torch.float64, device="cuda")
    dim = mesh["dim"]
    prev = None
    for call, steps in enumerate((3, 0, 2)):
        sim.step(steps)
        sim.totals_noalloc(out.data_ptr())
        sim.sync()
        torch.cuda.synchronize()
        got = out.cpu().numpy().copy()
        exp = _expected(sim.moments(fields=False), dim)
        assert np.all(np.isfinite(got)), call
        assert np.abs(got - exp).max() <= 1e-12 * exp[0], (call, got, exp)
        if steps == 0:
            # a repeated call on an unchanged state gives the identical result
            assert np.array_equal(got, prev)
        prev = got


def test_totals_noalloc_rejects_null_output():
    V = _lib()
    mesh = W.periodic_sine_mesh(8, 0.02)
    rho, u = W.taylor_green_fields(mesh, L=8)
    sim = V.Sim(V.Mesh(mesh), W.params(0.8), rho, u)
    with pytest.raises(V.VlbError) as e:
        sim.totals_noalloc(0)
    assert e.value.code == "EINVAL"


def test_totals_noalloc_runs_on_the_mesh_device():
    """Called with another device current, the call still runs on the mesh's
    device (whose scratch address it uses) and leaves the caller's device
    current. Needs two GPUs."""
    torch = pytest.importorskip("torch")
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two visible GPUs")
    V = _lib()
    torch.cuda.set_device(0)
    mesh = W.channel_mesh(16, 12, 8, stretch=0.7, bump=0.05)
    rho, u = W.noise_fields(mesh, amp=0.01, seed=2)
    sim = V.Sim(V.Mesh(mesh), W.params(0.8), rho, u, precision=V.VLB_F64)
    sim.step(2)
    out = torch.full((7,), float("nan"), dtype=torch.float64, device="cuda:0")
    torch.cuda.set_device(1)
    sim.totals_noalloc(out.data_ptr())
    assert torch.cuda.current_device() == 1
    torch.cuda.set_device(0)
    sim.sync()
    torch.cuda.synchronize(0)
    exp = _expected(sim.moments(fields=False), 3)
    assert np.abs(out.cpu().numpy() - exp).max() <= 1e-12 * exp[0]
