"""Pins of the oracle's body force and wall geometry, each against something
other than the oracle's own formula.

The body force is not in the paper; the oracle adds rho G . g^i to F^i of
Eq. 27 inside the fixed point (G Euclidean). What fixes it independently:

  - momentum: with the force, sum_a e_a(q) deltaN_a = J chi + J rho G per cell
    (g_i (G . g^i) = G), so the invariant M(t) of Eqs. 23-27 grows by exactly
    G times the total mass every step on any periodic mesh (the inertial part
    telescopes as without the force);
  - a uniform state on a periodic affine mesh stays uniform (Theta = 0), and
    its moments then follow in closed form from Eqs. 14-17, 20, 31 and 32:
    rho U^i grows by rho G^i per step, and the second moment relaxes as
    Pi <- Pi - (Pi - Pi^eq)/tau with Pi^eq = rho T0 g^ij + rho U~^i U~^j and
    U~ = U + F / (2 rho) (text after Eq. 32);
  - Poiseuille flow in a sheared (non-orthogonal) channel: the bulk profile is
    the parabola of nu = (tau - 1/2) T0 (Eq. 88) with curvature G / (2 nu)
    exactly, and the wall slip of halfway bounce-back shrinks at second order.

Each plausible slip in the term (g_i in place of g^i, rho dropped, G counted
again inside U~) is planted in a compiled copy of the oracle and must fail
one of these pins.

Walls (also not in the paper): ghost nodes are linear extrapolations, so on
an affine mesh with wall axes every cell, wall rows included, has the affine
closed form (g_i = A e_i, J = det A, g^ij = (A^T A)^-1, Theta = 0 in both
readings of the wall links), and on a polar mesh with walls at constant radius
the ghost nodes fall exactly on the polar grid, so Theta on the links that
cross a wall (wall_links = 1) equals the polar closed form.
"""
import math

import numpy as np
import pytest

from oracle import OracleSim, cell_geometry, lattice
from oracle.build import SRC, build_oracle_copy
from oracle.vlbo import OracleError, load_library
from paper_2401_17183_gb300 import workloads as W

T0 = 1.0 / 3.0


# ---------------------------------------------------------------------------- meshes

def _sheared_channel(N, n0=2, s=0.2, h=0.9):
    """2D channel, axis 0 periodic (streamwise), axis 1 walls: x = i + s j,
    y = h j; the walls sit at j = -1/2 and j = N - 1/2."""
    i = np.arange(n0, dtype=float)
    j = np.arange(N, dtype=float)
    I, Jj = np.meshgrid(i, j, indexing="ij")
    X = np.stack([I + s * Jj, h * Jj], -1)[:, :, None, :]
    return W._mesh(2, (n0, N, 1), X, (W.PERIODIC, W.WALL), shift=[[n0, 0], [0, 0]])


def _affine_walls(A, n, wall_axis, wall_links):
    """Affine mesh x = A q with walls on one axis, periodic elsewhere."""
    A = np.asarray(A, dtype=float)
    D = A.shape[0]
    n3 = tuple(n) + (1,) * (3 - len(n))
    Q = np.stack(np.meshgrid(*[np.arange(n3[a], dtype=float) for a in range(D)], indexing="ij"), -1)
    X = Q @ A.T
    bc = [W.WALL if a == wall_axis else W.PERIODIC for a in range(D)]
    shift = [A[:, a] * n3[a] if a != wall_axis else np.zeros(D) for a in range(D)]
    return W._mesh(D, n3, X, bc, shift=shift, wall_links=wall_links)


# ---------------------------------------------------------------------------- pins

def _M_growth_error(mesh, G, steps=200, lib=None):
    """| M(t) - M(0) - t G mass | / | t G mass | on a periodic mesh."""
    D = mesh["dim"]
    bf = tuple(G) + (0.0,) * (3 - D)
    rho, u = W.noise_fields(mesh, amp=0.02, seed=3, rho_amp=0.01)
    o = OracleSim(mesh, W.params(0.8, body_force=bf), lib=lib)
    o.init(rho, u)
    m0 = o.moments()
    o.step(steps)
    m1 = o.moments()
    pred = steps * np.asarray(G) * m0["mass"]
    return (np.abs(m1["M"] - m0["M"] - pred).max() / np.abs(pred).max(),
            abs(m1["mass"] - m0["mass"]) / m0["mass"])


def _uniform_acceleration_error(A, G, rho0=1.2, tau=0.7, steps=12, lib=None):
    """Largest deviation of the oracle's uniform state from the closed form,
    relative to the moment's own size (U and the second moment Pi)."""
    A = np.asarray(A, dtype=float)
    D = A.shape[0]
    q = 9 if D == 2 else 19
    mesh = W.affine_mesh(A, (4, 3, 3)[:D])
    nc = W.ncell(mesh)
    U0 = np.array([0.01, -0.02, 0.015])[:D]
    u0 = A @ U0                                # Euclidean u = U^i g_i, g_i = A e_i
    o = OracleSim(mesh, W.params(tau, body_force=tuple(G) + (0.0,) * (3 - D)), lib=lib)
    o.init(np.full(nc, rho0), np.tile(u0, (nc, 1)))
    c, _, _ = lattice(q)
    c = c[:, :D].astype(float)
    J = abs(np.linalg.det(A))
    ginv = np.linalg.inv(A.T @ A)              # g^ij
    Gi = np.linalg.solve(A, np.asarray(G))     # G^i = G . g^i, g^i the rows of A^-1
    U = U0.copy()
    Pi = rho0 * T0 * ginv + rho0 * np.outer(U0, U0)
    err_u = err_p = 0.0
    for t in range(steps):
        Ut = U + 0.5 * Gi                      # U~ = U + F / (2 rho), F = rho G^i
        Pieq = rho0 * T0 * ginv + rho0 * np.outer(Ut, Ut)
        Pi = Pi - (Pi - Pieq) / tau
        U = U + Gi
        o.step(1)
        N = o.get_state()                      # (q, ncell)
        f = N / J
        rho = f.sum(0)
        Uo = (c.T @ f) / rho                   # (D, ncell)
        Po = np.einsum("ai,aj,an->ijn", c, c, f)
        assert np.abs(rho - rho0).max() < 1e-14
        err_u = max(err_u, np.abs(Uo - U[:, None]).max() / np.abs(U).max())
        err_p = max(err_p, np.abs(Po - Pi[:, :, None]).max() / np.abs(Pi).max())
    return err_u, err_p


A2 = [[1.1, 0.25], [-0.1, 0.9]]
A3 = [[1.1, 0.2, -0.1], [0.05, 0.9, 0.15], [-0.1, 0.1, 1.05]]


@pytest.mark.parametrize("case", ["sine2d", "sine3d"])
def test_momentum_invariant_grows_by_body_force_times_mass(case):
    if case == "sine2d":
        mesh, G = W.periodic_sine_mesh(16, 0.02), (2e-5, -1e-5)
    else:
        mesh, G = W.periodic_sine_mesh3d(8, 0.02), (2e-5, -1e-5, 1.5e-5)
    e_M, e_mass = _M_growth_error(mesh, G)
    assert e_M <= 1e-12, e_M
    assert e_mass <= 1e-13, e_mass


@pytest.mark.parametrize("A", [A2, A3], ids=["d2q9", "d3q19"])
def test_uniform_acceleration_on_affine_mesh(A):
    G = (1e-3, -6e-4, 8e-4)[:len(A)]
    e_u, e_p = _uniform_acceleration_error(A, G)
    assert e_u <= 1e-13 and e_p <= 1e-13, (e_u, e_p)


def test_poiseuille_in_sheared_channel():
    tau, G, h, s = 0.8, 1e-6, 0.9, 0.2
    nu = (tau - 0.5) * T0
    slips = []
    for N in (16, 32):
        mesh = _sheared_channel(N, s=s, h=h)
        X = W.node_positions(mesh)
        y = X[:, 1]
        qy = (y + h / 2) * (h * (N - 0.5) - y)          # (y - y_lo)(y_hi - y)
        exact = G / (2 * nu) * qy
        u0 = np.zeros_like(X)
        u0[:, 0] = exact
        o = OracleSim(mesh, W.params(tau, body_force=(G, 0, 0)))
        o.init(np.ones(len(y)), u0)
        # twelve viscous time constants of the slowest mode
        o.step(int(12 * (N * h) ** 2 / (nu * math.pi ** 2)))
        ut = o.moments()["u_tilde"]
        umax = exact.max()
        # the flow is along the walls
        assert np.abs(ut[:, 1]).max() <= 1e-9 * umax
        # bulk: exactly the parabola of nu = (tau - 1/2) T0 with curvature G / (2 nu)
        Afit = np.stack([qy, np.ones_like(qy)], 1)
        coef = np.linalg.lstsq(Afit, ut[:, 0], rcond=None)[0]
        assert abs(coef[0] / (G / (2 * nu)) - 1) <= 1e-6, coef
        assert np.abs(Afit @ coef - ut[:, 0]).max() <= 1e-7 * umax
        slips.append(coef[1] / umax)
    # the halfway bounce-back slip converges at second order
    ratio = slips[0] / slips[1]
    assert 3.8 <= ratio <= 4.2, slips
    assert abs(slips[1]) <= 2e-3, slips


# ---------------------------------------------------------------------------- planted mistakes

MUTATIONS = {
    # the basis: G . g_i in place of G . g^i
    "g_low_in_place_of_g_up": ("out->G[i] = prm ? dot3(prm->body_force, out->g_up[i]) : 0.0;",
                               "out->G[i] = prm ? dot3(prm->body_force, out->g_low[i]) : 0.0;"),
    # rho dropped from rho G^i
    "rho_dropped": ("Fnew[i] = JF / J + rho * cell->G[i];", "Fnew[i] = JF / J + cell->G[i];"),
    # G counted once more inside U~
    "counted_again_in_Ut": ("for (int i = 0; i < D; i++) Ut[i] = U[i] + 0.5 * (F[i] / rho);",
                            "for (int i = 0; i < D; i++) Ut[i] = U[i] + 0.5 * (F[i] / rho) + 0.5 * cell->G[i];"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_body_force_mistakes_fail_the_pins(name, tmp_path):
    src = open(SRC).read()
    good, bad = MUTATIONS[name]
    assert src.count(good) == 1, "the oracle line this mutation targets has changed"
    lib = load_library(build_oracle_copy(src.replace(good, bad), str(tmp_path)))
    e_M, _ = _M_growth_error(W.periodic_sine_mesh(16, 0.02), (2e-5, -1e-5), lib=lib)
    e_u, e_p = _uniform_acceleration_error(A2, (1e-3, -6e-4), lib=lib)
    # every pin passes at <= 1e-12 on the real oracle; each mistake breaks one by far more
    assert max(e_M, e_u, e_p) > 1e-8, (e_M, e_u, e_p)


# ---------------------------------------------------------------------------- wall geometry

@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("wall_links", [0, 1])
def test_affine_mesh_with_walls_closed_form(D, wall_links):
    A = np.array(A2 if D == 2 else A3)
    n = (4, 3) if D == 2 else (3, 4, 3)
    wall_axis = 1
    mesh = _affine_walls(A, n, wall_axis, wall_links)
    q = 9 if D == 2 else 19
    c, _, _ = lattice(q)
    ginv = np.linalg.inv(A.T @ A)
    cells = [tuple(idx) + (0,) * (3 - D) for idx in np.ndindex(*n)]
    for qi in cells:
        g = cell_geometry(mesh, qi)
        assert np.allclose(g["g_low"][:D, :D], A.T, atol=1e-14), qi
        assert abs(g["J"] - np.linalg.det(A)) < 1e-14
        assert np.allclose(g["ginv"][:D, :D], ginv, atol=1e-13)
        assert np.abs(g["theta"]).max() < 1e-14, qi
        for a in range(q):
            p = qi[wall_axis] + c[a][wall_axis]
            assert g["wall_link"][a] == (1 if (p < 0 or p >= n[wall_axis]) else 0), (qi, a)


def _polar_theta(r, dr, dth, ca, cb):
    """Theta^i_j(q + c, q) on the polar grid r_i = r0 + i dr, theta_j = j dth,
    for a link (ca, cb) in index space (closed form of Eqs. 1, 3, 7, 11)."""
    s = math.sin(dth / 2)
    rp = r + ca * dr
    return np.array([[math.cos(cb * dth) - 1.0, -2 * rp * s * math.sin(cb * dth) / dr],
                     [dr * math.sin(cb * dth) / (2 * r * s), (rp / r) * math.cos(cb * dth) - 1.0]])


@pytest.mark.parametrize("wall_links", [0, 1])
def test_polar_walls_ghost_geometry_closed_form(wall_links):
    nr, nth, R1, R2, dth = 6, 4, 20.0, 26.0, 0.05
    mesh = W.polar_mesh(nr, nth, R1, R2, dtheta=dth, wall_links=wall_links)
    dr = (R2 - R1) / nr
    c, _, _ = lattice(9)
    s = math.sin(dth / 2)
    for i in (0, 1, nr - 2, nr - 1):
        for j in range(nth):
            g = cell_geometry(mesh, (i, j, 0))
            r, th = R1 + (i + 0.5) * dr, j * dth
            rh = np.array([math.cos(th), math.sin(th), 0])
            thh = np.array([-math.sin(th), math.cos(th), 0])
            assert np.allclose(g["g_low"][0], dr * rh, atol=1e-13)
            assert np.allclose(g["g_low"][1], 2 * r * s * thh, atol=1e-12)
            for a in range(9):
                crosses = not (0 <= i + c[a][0] < nr)
                assert g["wall_link"][a] == int(crosses)
                th_a = g["theta"][a][:2, :2]
                if crosses and wall_links == 0:
                    assert np.abs(th_a).max() == 0.0
                else:
                    ex = _polar_theta(r, dr, dth, c[a][0], c[a][1])
                    assert np.allclose(th_a, ex, atol=1e-12, rtol=1e-12), (i, j, a, th_a, ex)


@pytest.mark.parametrize("wall_links", [0, 1])
def test_walls_across_a_uniform_axis(wall_links):
    """Walls across an axis of uniform spacing (the spanwise axis of the
    bumped, stretched channel, which is the fastest axis): the extrapolated
    ghost nodes continue the uniform spacing, so J and g^ij are the same in
    every cell of a row, and so is every Theta when wall-crossing links take
    their Theta from the ghosts (wall_links = 1); with wall_links = 0 those
    links carry Theta = 0 instead, while the interior cells of the row keep
    the (non-zero) value that the ghosts would give."""
    n = (8, 6, 5)
    mesh = dict(W.channel_mesh(*n, stretch=0.7, bump=0.05, wall_links=wall_links))
    mesh["bc"] = (W.PERIODIC, W.WALL, W.WALL)
    shift = mesh["shift"].copy()
    shift[2] = 0.0
    mesh["shift"] = shift
    g = OracleSim(mesh, W.params(0.8)).geometry()
    J = g["J"].reshape(n)
    ginv = g["ginv"].reshape(n + (-1,))
    th = g["theta"].reshape(n + (19, 3, 3))
    wl = g["wall_link"].reshape(n + (19,))
    c, _, _ = lattice(19)
    cz = np.array([c[a][2] for a in range(19)])
    mid = n[2] // 2
    assert np.abs(J - J[:, :, mid:mid + 1]).max() < 1e-14
    assert np.abs(ginv - ginv[:, :, mid:mid + 1]).max() < 1e-14
    for z, crossing in ((0, cz < 0), (n[2] - 1, cz > 0)):
        assert (wl[:, :, z][:, :, crossing] == 1).all()
        inner = th[:, :, mid][:, :, crossing]
        assert np.abs(inner).max() > 0.05   # the readings differ on this mesh
        got = th[:, :, z][:, :, crossing]
        if wall_links:
            assert np.abs(got - inner).max() < 1e-14
        else:
            assert np.abs(got).max() == 0.0
        # links that stay inside the row agree in both readings
        assert np.abs(th[:, :, z][:, :, ~crossing] - th[:, :, mid][:, :, ~crossing]).max() < 1e-14


WALL_MUTATIONS = {
    # the ghost node behind a wall copies the wall-row node instead of
    # extrapolating linearly from the two rows inside
    "ghost_copies_the_wall_row": ("for (int d = 0; d < 3; d++) out[d] = 2.0 * y[d] - z[d];",
                                  "for (int d = 0; d < 3; d++) out[d] = y[d];"),
    # the extrapolation below the lower wall skips a row
    "ghost_stencil_skips_a_row": ("r2[a] = p[a] + 2;", "r2[a] = p[a] + 3;"),
}


def _wall_geometry_error(lib, wall_links):
    """Largest deviation of g_i, J and Theta from the affine closed form on a 3D
    affine mesh with walls on one axis (every cell, wall rows included)."""
    A = np.array(A3)
    n = (3, 4, 3)
    g = OracleSim(_affine_walls(A, n, 1, wall_links), W.params(0.8), lib=lib).geometry()
    e_g = np.abs(g["g_low"][:, :3, :3] - A.T[None]).max()
    e_J = np.abs(g["J"] - np.linalg.det(A)).max()
    return max(e_g, e_J, np.abs(g["theta"]).max())


@pytest.mark.parametrize("wall_links", [0, 1])
@pytest.mark.parametrize("name", sorted(WALL_MUTATIONS))
def test_planted_wall_geometry_mistakes_fail_the_pins(name, wall_links, tmp_path):
    assert _wall_geometry_error(None, wall_links) < 1e-13
    src = open(SRC).read()
    good, bad = WALL_MUTATIONS[name]
    assert src.count(good) == 1, "the oracle line this mutation targets has changed"
    lib = load_library(build_oracle_copy(src.replace(good, bad), str(tmp_path)))
    # caught either by the closed form or, where the mistake makes a degenerate
    # cell (a ghost on top of a node), by the oracle refusing the mesh
    try:
        err = _wall_geometry_error(lib, wall_links)
    except OracleError as e:
        assert "EGEOM" in str(e)
        return
    assert err > 1e-3
