"""GPU parity: the CUDA path (through the C-ABI) against the FP64 CPU oracle on
the same seeded inputs.

Tolerances: FP64 mode <= 1e-12 relative; FP32 mode <= 2e-5 max relative on
rho and u (u normalised by max|u|); the geometry precompute <= 1e-13.
"""
import math

import numpy as np
import pytest

from oracle import OracleSim, cell_geometry, collide, equilibrium
from oracle import lattice as olat
from paper_2401_17183_gb300 import workloads as W

from .helpers import oracle_state_in_lib_order, perm, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session")
def V():
    from paper_2401_17183_gb300 import build as B
    B.build()
    from paper_2401_17183_gb300 import vlb
    vlb.load()
    return vlb


def _wavy3d(n=(6, 5, 4), amp=0.08, seed=7):
    rng = np.random.default_rng(seed)
    q = np.stack(np.meshgrid(*[np.arange(k) for k in n], indexing="ij"), -1)
    A = np.array([[1.1, 0.15, 0.05], [-0.1, 0.9, 0.1], [0.05, -0.05, 1.2]])
    X = q @ A.T
    for d in range(3):
        for _ in range(2):
            k = rng.integers(-1, 2, size=3)
            ph = rng.uniform(0, 2 * np.pi)
            X[..., d] += amp * np.sin(2 * np.pi * (k[0] * q[..., 0] / n[0] + k[1] * q[..., 1] / n[1]
                                                   + k[2] * q[..., 2] / n[2]) + ph)
    return W._mesh(3, n, X, (0, 0, 0), shift=[A[:, a] * n[a] for a in range(3)])


MESHES = {
    "sine32": lambda: W.periodic_sine_mesh(32, 0.02),
    "sine16_literal": lambda: W.periodic_sine_mesh(16, 0.1),
    "channel_tanh2.5": lambda: W.channel_mesh(12, 10, 6, stretch=2.5, bump=0.05),
    "channel_tanh0.7": lambda: W.channel_mesh(10, 8, 5, stretch=0.7, bump=0.05),
    "channel_ghost_links": lambda: W.channel_mesh(10, 8, 5, stretch=0.7, bump=0.05, wall_links=1),
    "wedge1": lambda: W.polar_mesh(8, 1, 40.0, 48.0, dtheta=1.0 / 44),
    "wedge3": lambda: W.polar_mesh(6, 3, 30.0, 36.0, dtheta=1.0 / 33),
    "wavy3d": lambda: _wavy3d(),
}


@pytest.mark.parametrize("name", sorted(MESHES))
def test_geometry_parity(V, name):
    mesh = MESHES[name]()
    q = mesh["q"]
    D = mesh["dim"]
    gm = V.Mesh(mesh).geometry()
    om = OracleSim(mesh, W.params(0.8)).geometry()
    co, _, _ = olat(q)
    cl, _ = V.lattice(q)
    p = perm(cl, co)   # library direction a is oracle direction p[a]
    assert rel_err(gm["J"], om["J"]) < 1e-13
    assert rel_err(gm["g_low"], om["g_low"][:, :D, :D]) < 1e-13
    assert rel_err(gm["ginv"], om["ginv"][:, :D, :D]) < 1e-13
    # K^i_a = sum_j c^j_a Theta^i_j(q + c_a, q)
    Ko = np.einsum("naij,aj->nai", om["theta"][:, :, :D, :D], co[:, :D].astype(float))
    Ko = Ko[:, p, :]
    scale = max(np.abs(Ko).max(), 1e-3)
    assert np.abs(gm["K"] - Ko).max() <= 1e-13 * scale


def _run_pair(V, mesh, prm, rho, u, steps_list, precision=None, coef_mode=0):
    """Return [(gpu_state, oracle_state_lib_order)] after each cumulative step count."""
    precision = V.VLB_F64 if precision is None else precision
    gm = V.Mesh(mesh)
    gs = V.Sim(gm, prm, rho, u, precision=precision, coef_mode=coef_mode)
    os_ = OracleSim(mesh, prm)
    os_.init(rho, u)
    co, _, _ = olat(mesh["q"])
    cl, _ = V.lattice(mesh["q"])
    out = []
    done = 0
    for s in steps_list:
        gs.step(s - done)
        os_.step(s - done)
        done = s
        out.append((gs.get_state(), oracle_state_in_lib_order(os_.get_state(), co, cl), gs, os_))
    return out


@pytest.mark.parametrize("case", ["sine_d2q9", "channel_d3q19", "channel_ghost_links",
                                  "wedge_moving_wall", "wavy3d"])
def test_aa_layout_first_steps(V, case):
    """Even and odd A-A steps (1, 2, 3 steps) against the oracle's two-array stream."""
    if case == "sine_d2q9":
        mesh = W.periodic_sine_mesh(12, 0.02)
        prm = W.params(0.7)
        rho, u = W.noise_fields(mesh, amp=0.03, seed=3, rho_amp=0.01)
    elif case in ("channel_d3q19", "channel_ghost_links"):
        mesh = W.channel_mesh(8, 6, 5, stretch=0.7, bump=0.05,
                              wall_links=1 if case == "channel_ghost_links" else 0)
        prm = W.params(0.6, body_force=(2e-5, 0, 0))
        rho, u = W.noise_fields(mesh, amp=0.01, seed=2)
    elif case == "wedge_moving_wall":
        mesh = W.polar_mesh(8, 1, 40.0, 48.0, dtheta=1.0 / 44)
        wo = np.zeros((3, 2, 3))
        wo[0, 0, 2] = 0.01 / 40
        wu = np.zeros((3, 2, 3))
        wu[0, 1, :2] = [0.001, -0.002]
        prm = W.params(0.9, wall_omega=wo, wall_u=wu)
        rho, u = W.noise_fields(mesh, amp=0.01, seed=4)
    else:
        mesh = _wavy3d()
        prm = W.params(0.8)
        rho, u = W.noise_fields(mesh, amp=0.02, seed=5, rho_amp=0.01)
    for g, o, _, _ in _run_pair(V, mesh, prm, rho, u, [1, 2, 3]):
        assert rel_err(g, o) < 1e-13


@pytest.mark.parametrize("nz", [128, 256])
def test_whole_tile_rows(V, nz):
    """Plane-mode meshes whose periodic fastest axis spans whole 128-cell
    tiles (one and two per row: the wrap-around of an odd step at both row
    ends inside one tile and across tiles): steps 1-3 and 41 against the
    oracle in FP64, and 41 steps in FP32."""
    mesh = W.channel_mesh(6, 5, nz, stretch=0.7, bump=0.05)
    prm = W.params(0.6, body_force=(2e-5, 0, 1e-5))
    rho, u = W.noise_fields(mesh, amp=0.01, seed=7)
    res = _run_pair(V, mesh, prm, rho, u, [1, 2, 3, 41], coef_mode=V.VLB_COEF_PLANE)
    assert res[0][2].layout()["plane"]
    for g, o, _, _ in res[:3]:
        assert rel_err(g, o) < 1e-13
    assert rel_err(res[3][0], res[3][1]) < 1e-12
    om = res[3][3].moments()
    g32 = V.Sim(V.Mesh(mesh), prm, rho, u, precision=V.VLB_F32, coef_mode=V.VLB_COEF_PLANE)
    g32.step(41)
    _cmp_moments(g32.moments(), om, 2e-5)


def _cmp_moments(gm, om, tol):
    assert rel_err(gm["rho"], om["rho"], 1.0) < tol
    su = np.abs(om["u"]).max()
    assert rel_err(gm["u"], om["u"], su) < tol
    assert rel_err(gm["u_tilde"], om["u_tilde"], su) < tol


@pytest.fixture(scope="module")
def config1_oracle():
    """64 x 64 D2Q9 periodic mapped box (amplitude 0.02 L), tau = 0.8,
    Taylor-Green 0.01 + 1e-4 noise, 1000 steps of the oracle."""
    mesh = W.periodic_sine_mesh(64, 0.02)
    prm = W.params(0.8)
    rho, u = W.taylor_green_fields(mesh)
    o = OracleSim(mesh, prm)
    o.init(rho, u)
    m0 = o.moments()
    o.step(1000)
    return mesh, prm, rho, u, m0, o.moments()


def test_config1_fp64_1000_steps(V, config1_oracle):
    mesh, prm, rho, u, m0, m1 = config1_oracle
    g = V.Sim(V.Mesh(mesh), prm, rho, u, precision=V.VLB_F64)
    g0 = g.moments()
    g.step(1000)
    gm = g.moments()
    _cmp_moments(gm, m1, 1e-12)
    assert abs(gm["mass"] - m1["mass"]) <= 1e-12 * m1["mass"]
    scale = np.abs(m1["u_tilde"]).sum()
    assert np.abs(gm["M"] - m1["M"]).max() <= 1e-12 * scale
    # the GPU's own invariants over the run
    assert abs(gm["mass"] - g0["mass"]) <= 1e-13 * g0["mass"]
    assert np.abs(gm["M"] - g0["M"]).max() <= 1e-12 * scale


def test_config1_fp32_1000_steps(V, config1_oracle):
    mesh, prm, rho, u, m0, m1 = config1_oracle
    g = V.Sim(V.Mesh(mesh), prm, rho, u, precision=V.VLB_F32)
    g.step(1000)
    gm = g.moments()
    _cmp_moments(gm, m1, 2e-5)


def test_config1_literal_mesh(V):
    """Amplitude 0.1 L (outside the realizable range): FP64 parity while the
    run is finite, then the GPU reports the failure as the oracle does."""
    mesh = W.periodic_sine_mesh(64, 0.1)
    prm = W.params(0.8)
    rho, u = W.taylor_green_fields(mesh)
    pairs = _run_pair(V, mesh, prm, rho, u, [1, 2, 3, 4])
    for g, o, _, _ in pairs:
        assert rel_err(g, o) < 1e-12
    gs = pairs[-1][2]
    with pytest.raises(V.VlbError) as e:
        for _ in range(40):
            gs.step(1)
            gs.sync()
            gs.moments(fields=False)
    assert e.value.code in ("ENOCONV", "ENONFINITE")


@pytest.fixture(scope="module")
def channel_oracle():
    """D3Q19 channel: 16 x 12 x 8, tanh stretching 0.7, lower-wall bump 0.05 h,
    walls on eta, body force along xi, tau = 0.6, 1% seeded velocity noise."""
    mesh = W.channel_mesh(16, 12, 8, stretch=0.7, bump=0.05)
    prm = W.params(0.6, body_force=(1e-5, 0, 0))
    rho, u = W.noise_fields(mesh, amp=0.01, seed=2)
    o = OracleSim(mesh, prm)
    o.init(rho, u)
    o.step(50)
    m50 = o.moments()
    o.step(150)
    return mesh, prm, rho, u, m50, o.moments()


def test_channel_fp64(V, channel_oracle):
    mesh, prm, rho, u, m50, _ = channel_oracle
    for mode in (V.VLB_COEF_FULL, V.VLB_COEF_PLANE):
        g = V.Sim(V.Mesh(mesh), prm, rho, u, precision=V.VLB_F64, coef_mode=mode)
        assert g.layout()["plane"] == (mode == V.VLB_COEF_PLANE)
        g.step(50)
        gm = g.moments()
        _cmp_moments(gm, m50, 1e-12)
        assert abs(gm["mass"] - m50["mass"]) <= 1e-12 * m50["mass"]


def test_channel_fp32(V, channel_oracle):
    mesh, prm, rho, u, _, m200 = channel_oracle
    for mode in (V.VLB_COEF_FULL, V.VLB_COEF_PLANE):
        g = V.Sim(V.Mesh(mesh), prm, rho, u, precision=V.VLB_F32, coef_mode=mode)
        g.step(200)
        _cmp_moments(g.moments(), m200, 2e-5)


@pytest.fixture(scope="module")
def bump3d_oracle():
    """D3Q19 channel whose lower-wall bump also varies spanwise (12 x 10 x 16,
    tanh stretching 0.7, bump 0.05 h): the geometry changes along every axis,
    so every cell has its own coefficient record and the step forms the rest
    state from J and g^ij. Walls on eta, body force along xi, tau = 0.8, 1%
    seeded velocity noise; 100 oracle steps."""
    mesh = W.channel_bump3d_mesh(12, 10, 16, stretch=0.7, bump=0.05)
    prm = W.params(0.8, body_force=(1e-5, 0, 0))
    rho, u = W.noise_fields(mesh, amp=0.01, seed=5)
    o = OracleSim(mesh, prm)
    o.init(rho, u)
    o.step(100)
    return mesh, prm, rho, u, o.moments()


@pytest.mark.parametrize("prec,tol", [("F64", 1e-12), ("F32", 2e-5)])
def test_general_mesh_against_the_oracle(V, bump3d_oracle, prec, tol):
    mesh, prm, rho, u, m100 = bump3d_oracle
    g = V.Sim(V.Mesh(mesh), prm, rho, u, precision=getattr(V, "VLB_" + prec))
    lay = g.layout()
    assert not lay["plane"] and lay["coef_per_cell"] == 136
    g.step(100)
    gm = g.moments()
    _cmp_moments(gm, m100, tol)
    if prec == "F64":
        assert abs(gm["mass"] - m100["mass"]) <= 1e-12 * m100["mass"]


@pytest.fixture(scope="module")
def channel_tiles_oracle():
    """D3Q19 channel whose periodic fastest axis is one whole 128-cell tile
    (4 x 5 x 128, plane mode): tanh wall-normal stretching 0.7 (J, g^ij and
    Theta vary across the channel), walls, body force along xi, tau = 0.6, 1%
    seeded velocity noise; 1000 oracle steps (about half a minute)."""
    mesh = W.channel_mesh(4, 5, 128, stretch=0.7, bump=0.0)
    prm = W.params(0.6, body_force=(2e-5, 0, 0))
    rho, u = W.noise_fields(mesh, amp=0.01, seed=11)
    o = OracleSim(mesh, prm)
    o.init(rho, u)
    o.step(1000)
    return mesh, prm, rho, u, o.moments()


def test_channel_fp32_1000_steps_whole_tiles(V, channel_tiles_oracle):
    """The FP32 D3Q19 kernel of the benchmark against the FP64 oracle after
    1000 steps (<= 2e-5 on rho and on u, u normalised by max|u|): even steps
    take the 16-byte row copies of whole tiles, odd steps the neighbour
    gathers, both with walls and a body force."""
    mesh, prm, rho, u, om = channel_tiles_oracle
    g = V.Sim(V.Mesh(mesh), prm, rho, u, precision=V.VLB_F32)
    assert g.layout()["plane"]
    g.step(1000)
    gm = g.moments()
    _cmp_moments(gm, om, 2e-5)
    assert abs(gm["mass"] - om["mass"]) <= 2e-5 * om["mass"]


def test_couette_on_gpu_matches_closed_form(V):
    """The GPU path on the narrow-gap wedge (128 radial cells) from rest, and a
    full annulus (FP32) started from the closed form."""
    nr, R1, R2 = 128, 2560.0, 2688.0
    dth = 2.0 / (R1 + R2)
    Om = 0.02 / R1
    wo = np.zeros((3, 2, 3))
    wo[0, 0, 2] = Om
    tau = 1.0
    nu = (tau - 0.5) / 3.0
    Tc = (R2 - R1) ** 2 / (nu * math.pi ** 2)
    A = -Om * R1 ** 2 / (R2 ** 2 - R1 ** 2)
    B = Om * R1 ** 2 * R2 ** 2 / (R2 ** 2 - R1 ** 2)

    def err(mesh, sim):
        X = W.node_positions(mesh)
        r = np.hypot(X[:, 0], X[:, 1])
        th = np.stack([-X[:, 1] / r, X[:, 0] / r], -1)
        ut = (sim.moments()["u_tilde"] * th).sum(-1)
        ex = A * r + B / r
        return np.linalg.norm(ut - ex) / np.linalg.norm(ex), r, th

    mesh = W.polar_mesh(nr, 1, R1, R2, dtheta=dth)
    rho, u = W.rest_fields(mesh)
    s = V.Sim(V.Mesh(mesh), W.params(tau, wall_omega=wo), rho, u, precision=V.VLB_F64)
    s.step(int(9 * Tc))
    e, _, _ = err(mesh, s)
    assert e <= 2e-3, e
    # full annulus: periodic in theta with no transform at all
    nth = int(round(2 * math.pi / dth))
    full = W.polar_mesh(nr, nth, R1, R2, dtheta=2 * math.pi / nth)
    X = W.node_positions(full)
    r = np.hypot(X[:, 0], X[:, 1])
    th = np.stack([-X[:, 1] / r, X[:, 0] / r], -1)
    u0 = (A * r + B / r)[:, None] * th
    s2 = V.Sim(V.Mesh(full), W.params(tau, wall_omega=wo), np.ones(len(r)), u0,
               precision=V.VLB_F32)
    s2.step(int(3 * Tc))
    e2, _, _ = err(full, s2)
    assert e2 <= 2e-3, e2


def _oracle_one_step(mesh, prm, rho, u, qi, cache):
    """Arrived populations and moments at cell qi after one step from the
    equilibrium initial state, computed by the oracle cell by cell."""
    q = mesh["q"]
    D = mesh["dim"]
    n = mesh["n"]
    c, w, _ = olat(q)
    opp = [int(np.where((c == -c[a]).all(1))[0][0]) for a in range(q)]

    def idx(p):
        return (p[0] * n[1] + p[1]) * n[2] + p[2]

    def post(p):
        key = tuple(p)
        if key not in cache:
            g = cell_geometry(mesh, p, prm)
            k = idx(p)
            U = np.zeros(3)
            U[:D] = g["g_up"][:D, :D] @ u[k]
            N0 = g["J"] * equilibrium(q, rho[k], U, U, g["ginv"])
            cache[key] = (g, collide(q, g, prm, N0)["Np"])
        return cache[key]

    gq, npq = post(qi)
    N = np.zeros(q)
    for a in range(q):
        src = [qi[d] - int(c[a][d]) for d in range(3)]
        wall = any(mesh["bc"][d] == 1 and not (0 <= src[d] < n[d]) for d in range(D))
        if wall:
            N[a] = npq[opp[a]]
        else:
            s = [src[d] % n[d] for d in range(3)]
            N[a] = post(s)[1][a]
    J = gq["J"]
    r = N.sum() / J
    U = (c[:, :D].T @ N) / (J * r)
    return r, U @ gq["g_low"][:D, :D]


def test_full_size_channel_sampled_cells(V):
    """256^3 D3Q19 FP32 channel (the benchmark workload and launch shape):
    after one step, sampled cells (walls, seams, corners, interior) against
    the oracle cell by cell; then mass over 20 steps."""
    mesh = W.channel_mesh(256, 256, 256, stretch=0.7, bump=0.05)
    prm = W.params(0.6, body_force=(1e-6, 0, 0))
    rho, u = W.noise_fields(mesh, amp=0.01, seed=2)
    g = V.Sim(V.Mesh(mesh), prm, rho, u, precision=V.VLB_F32)
    assert g.layout()["plane"]
    g.step(1)
    gm = g.moments()
    rng = np.random.default_rng(0)
    picks = [(0, 0, 0), (255, 255, 255), (0, 255, 0), (255, 0, 255), (128, 0, 17), (7, 255, 200),
             (0, 128, 255), (255, 1, 0)]
    picks += [tuple(int(v) for v in rng.integers(0, 256, 3)) for _ in range(24)]
    cache = {}
    n = mesh["n"]
    umax = np.abs(u).max()
    for p in picks:
        r, uu = _oracle_one_step(mesh, prm, rho, u, p, cache)
        k = (p[0] * n[1] + p[1]) * n[2] + p[2]
        assert abs(gm["rho"][k] - r) < 2e-5, p
        assert np.abs(gm["u"][k] - uu).max() < 2e-5 * umax, p
    m0 = gm["mass"]
    g.step(20)
    m1 = g.moments(fields=False)
    assert abs(m1["mass"] - m0) < 1e-6 * m0


def test_state_roundtrip_and_reset(V):
    mesh = W.channel_mesh(8, 6, 4, stretch=0.7, bump=0.05)
    prm = W.params(0.7)
    rho, u = W.noise_fields(mesh, amp=0.01, seed=8)
    g = V.Sim(V.Mesh(mesh), prm, rho, u, precision=V.VLB_F64)
    g.step(3)
    N = g.get_state()
    assert g.time() == 3
    g.set_state(N)
    assert g.time() == 0
    assert np.array_equal(g.get_state(), N)
    g.reset(rho, u)
    o = OracleSim(mesh, prm)
    o.init(rho, u)
    co, _, _ = olat(19)
    cl, _ = V.lattice(19)
    assert rel_err(g.get_state(), oracle_state_in_lib_order(o.get_state(), co, cl)) < 1e-14


def test_error_paths(V):
    mesh = W.periodic_sine_mesh(8, 0.0)
    X = mesh["x"].copy()
    X[4, 3, 0] = X[2, 3, 0]
    bad = W._mesh(2, (8, 8, 1), X, (0, 0), shift=[[8, 0], [0, 8]])
    with pytest.raises(V.VlbError) as e:
        V.Mesh(bad)
    assert e.value.code == "EGEOM"
    good = V.Mesh(W.periodic_sine_mesh(16, 0.02))
    rho, u = W.taylor_green_fields(W.periodic_sine_mesh(16, 0.02), L=16)
    with pytest.raises(V.VlbError) as e:
        V.Sim(good, W.params(0.5), rho, u)
    assert e.value.code == "EINVAL"
    s = V.Sim(good, W.params(0.8, max_iter=1), rho, u)
    s.step(2)
    with pytest.raises(V.VlbError) as e:
        s.sync()
    assert e.value.code == "ENOCONV"
    # the context stays usable after a reported kernel error
    s2 = V.Sim(good, W.params(0.8), rho, u)
    s2.step(2)
    s2.sync()
    # a non-finite population, injected on the host through the state, is reported
    s3 = V.Sim(good, W.params(0.8), rho, u)
    N = s3.get_state()
    N[3, 17] = np.nan
    s3.set_state(N)
    s3.step(1)
    with pytest.raises(V.VlbError) as e:
        s3.sync()
    assert e.value.code in ("ENOCONV", "ENONFINITE")


def test_64bit_offsets_match_tiled_short_mesh(V):
    """A mesh with Q x ncell >= 2^31 (117 M cells, D3Q19 FP32, plane mode)
    runs the kernels with 64-bit offsets. Its initial fields repeat along the
    periodic fastest axis with period 8 and its geometry does not vary along
    it, so after every step its fields must equal, bit for bit, those of the
    8 x 8 x 8 mesh with the same fields (32-bit offsets) tiled along that
    axis: after an even and after an odd step of the A-A scheme."""
    n2 = 14336 * 128
    assert 19 * 8 * 8 * n2 >= 2 ** 31
    small = W.channel_mesh(8, 8, 8, stretch=0.7, bump=0.05)
    prm = W.params(0.8, body_force=(1e-5, 0, 0))
    rho_s, u_s = W.noise_fields(small, amp=0.01, seed=9)
    gs = V.Sim(V.Mesh(small), prm, rho_s, u_s, precision=V.VLB_F32)
    big = W.channel_mesh(8, 8, n2, stretch=0.7, bump=0.05)
    reps = n2 // 8
    rho_b = np.tile(rho_s.reshape(8, 8, 1, 8), (1, 1, reps, 1)).reshape(-1)
    u_b = np.tile(u_s.reshape(8, 8, 1, 8, 3), (1, 1, reps, 1, 1)).reshape(-1, 3)
    mb_mesh = V.Mesh(big)
    del big
    gb = V.Sim(mb_mesh, prm, rho_b, u_b, precision=V.VLB_F32)
    del rho_b, u_b
    assert gb.layout()["plane"] and gs.layout()["plane"]
    for parity in ("even", "odd"):
        gs.step(1)
        gb.step(1)
        ms, mb = gs.moments(), gb.moments()
        for key, shape in (("rho", (8, 8, 1, 8)), ("u", (8, 8, 1, 8, 3)), ("u_tilde", (8, 8, 1, 8, 3))):
            small_f = ms[key].reshape(shape)
            big_f = mb[key].reshape((8, 8, reps, 8) + shape[4:])
            assert np.array_equal(big_f, np.broadcast_to(small_f, big_f.shape)), (parity, key)
        del mb
    gb.close()
    mb_mesh.close()
