"""Batches: many simulations advanced by one kernel launch per time step.

The batch kernel runs the same per-cell code as vlb_step, only the
assignment of tiles to blocks differs, so a batch must reproduce the
members' individual time steps bit for bit: uneven D3Q19 channels in plane
mode (ragged fastest axis included), D2Q9 meshes in full mode in FP64,
whole 32-step graph replays plus remainders, a start at odd parity, and the
run-length tuner. Members that cannot share a launch are rejected.
"""
import numpy as np
import pytest

from paper_2401_17183_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    from paper_2401_17183_gb300 import build as B
    B.build()
    from paper_2401_17183_gb300 import vlb
    vlb.load()
    return vlb


def _channels(V, prec=None):
    sims = []
    for i, n in enumerate([(16, 12, 8), (24, 16, 130), (8, 6, 5), (32, 32, 40)]):
        mesh = W.channel_mesh(*n, stretch=0.7, bump=0.05)
        rho, u = W.noise_fields(mesh, amp=0.01, seed=10 + i)
        sims.append(V.Sim(V.Mesh(mesh), W.params(0.8, body_force=(1e-5, 0, 0)), rho, u,
                          precision=V.VLB_F32 if prec is None else prec))
    return sims


def _d2q9_full(V):
    meshes = [W.periodic_sine_mesh(16, 0.02), W.periodic_sine_mesh(40, 0.02),
              W.polar_mesh(16, 3, 300.0, 316.0, dtheta=1.0 / 308), W.periodic_sine_mesh(24, 0.01)]
    sims = []
    for i, mesh in enumerate(meshes):
        rho, u = W.noise_fields(mesh, amp=0.005, seed=20 + i)
        sims.append(V.Sim(V.Mesh(mesh), W.params(0.9), rho, u, precision=V.VLB_F64))
    return sims


@pytest.mark.parametrize("kind", ["d3q19_f32_plane", "d2q9_f64_full"])
def test_batch_matches_individual_steps(V, kind):
    make = _channels if kind.startswith("d3q19") else _d2q9_full
    alone, batched = make(V), make(V)
    assert batched[0].layout()["plane"] == (kind.endswith("plane"))
    b = V.Batch(batched)
    lay = b.layout()
    assert lay["blocks"] >= len(batched)
    steps = 70                      # two 32-step graph replays and a remainder
    for s in alone:
        s.step(steps)
    b.step(steps)
    for s, t in zip(alone, batched):
        t.sync()
        assert t.time() == s.time() == steps
        assert np.array_equal(s.get_state(), t.get_state())


def test_batch_from_odd_parity_and_tuner(V):
    alone, batched = _channels(V), _channels(V)
    for s in alone + batched:
        s.step(1)
    b = V.Batch(batched)
    run = b.tune(3)                 # advances every member by 4 x 3 steps
    assert run >= 1 and b.layout()["run_length"] == run
    b.step(40)
    for s in alone:
        s.step(12 + 40)
    for s, t in zip(alone, batched):
        assert t.time() == s.time() == 53
        assert np.array_equal(s.get_state(), t.get_state())


def test_batch_rejects_mixed_members(V):
    ch = _channels(V)[:2]
    d2 = _d2q9_full(V)[:1]
    with pytest.raises(V.VlbError) as e:
        V.Batch(ch + d2)
    assert e.value.code == "EINVAL"
    ch[1].step(1)                   # parities differ
    with pytest.raises(V.VlbError) as e:
        V.Batch(ch)
    assert e.value.code == "EINVAL"
    h = _channels(V, prec=V.VLB_F16)[:1]
    with pytest.raises(V.VlbError) as e:
        V.Batch(h)
    assert e.value.code == "EINVAL"
