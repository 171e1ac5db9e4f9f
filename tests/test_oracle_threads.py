"""The oracle's time step on several threads gives the same populations,
bit for bit, as on one (each cell reads its own arrivals and writes locations
no other cell writes), including the conservation totals. Walls, a body force
and a curved mesh are all present."""
import numpy as np

from oracle import OracleSim, set_threads
from paper_2401_17183_gb300 import workloads as W


def _run(nthreads, mesh, prm, rho, u, steps):
    set_threads(nthreads)
    o = OracleSim(mesh, prm)
    o.init(rho, u)
    o.step(steps)
    return o.get_state(), o.moments()


def test_threads_reproduce_one_thread_bit_for_bit():
    mesh = W.channel_mesh(12, 10, 9, stretch=0.7, bump=0.05)
    prm = W.params(0.8, body_force=(1e-5, 0.0, 0.0))
    rho, u = W.noise_fields(mesh, amp=0.01, seed=7)
    before = set_threads(0)
    try:
        N1, m1 = _run(1, mesh, prm, rho, u, 6)
        N4, m4 = _run(4, mesh, prm, rho, u, 6)
    finally:
        set_threads(before)
    assert np.array_equal(N1, N4)
    assert m1["mass"] == m4["mass"]
    assert np.array_equal(m1["M"], m4["M"])
    assert np.array_equal(m1["u_tilde"], m4["u_tilde"])
