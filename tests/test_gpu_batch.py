"""Batches: many simulations advanced by one kernel launch per time step.

The batch kernel runs the same per-cell code as vlb_step, only the
assignment of tiles to blocks differs, so a batch must reproduce the
members' individual time steps bit for bit: uneven D3Q19 channels in plane
mode (ragged fastest axis included), D2Q9 meshes in full mode in FP64,
whole 32-step graph replays plus remainders, a start at odd parity, and the
run-length tuner. Members that cannot share a launch are rejected. Each
member of an uneven D2Q9 batch is also held to the FP64 oracle itself: at
1e-12 in FP64 and at 2e-5 (rho, and u normalised by max|u|) in FP32.
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
    adv = b.tune_steps(3)
    run = b.tune(3)                 # every block shape and run length, 3 steps each
    lay = b.layout()
    assert run >= 1 and lay["run_length"] == run
    assert adv == 4 * 4 * 3 and lay["threads"] in (64, 128)
    b.step(40)
    for s in alone:
        s.step(adv + 40)
    for s, t in zip(alone, batched):
        assert t.time() == s.time() == 1 + adv + 40
        assert np.array_equal(s.get_state(), t.get_state())


@pytest.mark.parametrize("shape", range(4))
def test_batch_every_block_shape_matches_individual_steps(V, shape):
    """Each block shape the tuner may pick (tile width 128 with three register
    budgets, or 64) gives the members' own steps bit for bit, ragged rows
    included."""
    alone, batched = _channels(V), _channels(V)
    b = V.Batch(batched)
    b.set_shape(shape)
    assert b.layout()["threads"] == (64 if shape == 3 else 128)
    for s in alone:
        s.step(37)
    b.step(37)                      # one 32-step graph replay and a remainder
    for s, t in zip(alone, batched):
        t.sync()
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


def _uneven_d2q9():
    """Uneven D2Q9 members: stretched 2D channels (walls, plane mode) of
    different sizes, one with a ragged fastest axis, driven by a body force."""
    meshes = [W.channel2d_mesh(12, 40, stretch=0.5), W.channel2d_mesh(20, 136, stretch=0.7),
              W.channel2d_mesh(8, 24, stretch=0.3), W.channel2d_mesh(16, 256, stretch=0.6)]
    out = []
    for i, mesh in enumerate(meshes):
        rho, u = W.noise_fields(mesh, amp=0.01, seed=40 + i)
        out.append((mesh, W.params(0.8, body_force=(0.0, 1e-5, 0.0)), rho, u))
    return out


@pytest.mark.parametrize("prec,tol", [("F64", 1e-12), ("F32", 2e-5)])
def test_batch_members_match_the_oracle(V, prec, tol):
    members = _uneven_d2q9()
    steps = 70                      # two 32-step graph replays and a remainder
    sims = [V.Sim(V.Mesh(m), prm, rho, u, precision=getattr(V, "VLB_" + prec))
            for (m, prm, rho, u) in members]
    b = V.Batch(sims)
    b.step(steps)
    for (mesh, prm, rho, u), s in zip(members, sims):
        s.sync()
        o = OracleSim(mesh, prm)
        o.init(rho, u)
        o.step(steps)
        om, gm = o.moments(), s.moments()
        su = np.abs(om["u"]).max()
        assert rel_err(gm["rho"], om["rho"], 1.0) < tol
        assert rel_err(gm["u"], om["u"], su) < tol
        assert rel_err(gm["u_tilde"], om["u_tilde"], su) < tol
