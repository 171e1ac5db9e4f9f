"""Pins of the oracle's geometry (section 2.1) against closed forms and identities.

Each test checks the oracle against something other than itself: exact
closed forms on affine and polar meshes, the algebraic identities the paper
states after Eqs. 6-8, and the continuum (Christoffel) limit of Eq. 11 given
by Eqs. 63-66.
"""
import math
import os

import numpy as np
import pytest

from oracle import cell_geometry, lattice
from oracle.vlbo import OracleError
from paper_2401_17183_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _wavy3d(n=(6, 5, 4), amp=0.08, seed=7):
    """Smooth periodic 3D mesh with random Fourier wiggles (right-handed)."""
    rng = np.random.default_rng(seed)
    n0, n1, n2 = n
    q = np.stack(np.meshgrid(np.arange(n0), np.arange(n1), np.arange(n2), indexing="ij"), -1)
    A = np.array([[1.1, 0.15, 0.05], [-0.1, 0.9, 0.1], [0.05, -0.05, 1.2]])
    X = q @ A.T
    for d in range(3):
        for _ in range(2):
            k = rng.integers(-1, 2, size=3)
            ph = rng.uniform(0, 2 * np.pi)
            X[..., d] += amp * np.sin(2 * np.pi * (k[0] * q[..., 0] / n0 + k[1] * q[..., 1] / n1
                                                   + k[2] * q[..., 2] / n2) + ph)
    shift = [A[:, a] * n[a] for a in range(3)]
    return W._mesh(3, n, X, (0, 0, 0), shift=shift)


def test_velocity_sets_match_paper_and_isotropy():
    # D3Q19 set of section 2.1 (golden fixture), D2Q9 its planar restriction
    c19, w19, T0 = lattice(19)
    gold = np.loadtxt(os.path.join(GOLDEN, "d3q19_velocities.txt"), dtype=int)
    assert sorted(map(tuple, c19)) == sorted(map(tuple, gold))
    c9, w9, _ = lattice(9)
    assert sorted(map(tuple, c9)) == sorted(t for t in map(tuple, gold) if t[2] == 0)
    assert T0 == pytest.approx(1.0 / 3.0, abs=0)
    d = np.eye(3)
    for c, w, D in ((c9, w9, 2), (c19, w19, 3)):
        c = c[:, :D].astype(float)
        dd = d[:D, :D]
        # Eq. 10 up to 4th order
        assert abs(w.sum() - 1) < 1e-15
        assert np.allclose(np.einsum("a,ai,aj->ij", w, c, c), T0 * dd, atol=1e-15)
        m4 = np.einsum("a,ai,aj,ak,al->ijkl", w, c, c, c, c)
        d4 = (np.einsum("ij,kl->ijkl", dd, dd) + np.einsum("ik,jl->ijkl", dd, dd)
              + np.einsum("il,jk->ijkl", dd, dd))
        assert np.allclose(m4, T0 ** 2 * d4, atol=1e-15)
        # odd moments vanish
        assert np.allclose(np.einsum("a,ai->i", w, c), 0, atol=1e-16)
        assert np.allclose(np.einsum("a,ai,aj,ak->ijk", w, c, c, c), 0, atol=1e-16)
        # and the 6th-order condition fails, as the paper says for D3Q19
        m6 = np.einsum("a,ai,aj,ak,al,am,an->ijklmn", w, c, c, c, c, c, c)
        assert abs(m6[(0,) * 6] - 15 * T0 ** 3) > 0.1


def test_identities_on_curved_3d_mesh():
    mesh = _wavy3d()
    for qi in [(0, 0, 0), (3, 2, 1), (5, 4, 3), (2, 0, 3)]:
        g = cell_geometry(mesh, qi)
        gl, gu = g["g_low"], g["g_up"]
        # g_i . g^j = delta (after Eq. 7)
        assert np.allclose(gl @ gu.T, np.eye(3), atol=1e-14)
        # det g_ij = J^2 (Eq. 6); g^ij = inverse of g_ij (after Eq. 8)
        assert abs(np.linalg.det(g["gij"]) - g["J"] ** 2) < 1e-13 * g["J"] ** 2
        assert np.allclose(g["gij"] @ g["ginv"], np.eye(3), atol=1e-13)
        assert np.allclose(g["gij"], gl @ gl.T, atol=1e-15)
        # J = (g1 x g2) . g3 (Eq. 5)
        assert abs(np.dot(np.cross(gl[0], gl[1]), gl[2]) - g["J"]) < 1e-14
        # |g_i| is the mean of the two arm lengths (Eq. 3 with beta)
        X = mesh["x"]
        from oracle import position
        x0 = position(mesh, qi)
        for i in range(3):
            e = np.zeros(3, dtype=int)
            e[i] = 1
            dp = position(mesh, np.array(qi) + e) - x0
            dm = position(mesh, np.array(qi) - e) - x0
            assert abs(np.linalg.norm(gl[i]) - 0.5 * (np.linalg.norm(dp) + np.linalg.norm(dm))) < 1e-14
            # direction along D_i - D_-i
            u = (dp - dm) / np.linalg.norm(dp - dm)
            assert np.allclose(gl[i] / np.linalg.norm(gl[i]), u, atol=1e-14)
        assert X.shape[-1] == 3


def test_beta_is_one_for_collinear_arms():
    # 1-D stretching: arms along xi are collinear, so g_xi = (D_+ - D_-)/2 (Eq. 3, beta = 1)
    n = 12
    xi = np.arange(n, dtype=float)
    x = xi + 0.3 * np.sin(2 * np.pi * xi / n)
    X = np.stack(np.meshgrid(x, np.arange(4.0), indexing="ij"), -1)[:, :, None, :]
    mesh = W._mesh(2, (n, 4, 1), X, (0, 0), shift=[[n, 0], [0, 4]])
    for i in range(n):
        g = cell_geometry(mesh, (i, 1, 0))
        half = 0.5 * (x[(i + 1) % n] + (n if i == n - 1 else 0) - x[i - 1] + (n if i == 0 else 0))
        assert abs(g["g_low"][0][0] - half) < 1e-14
        assert abs(g["g_low"][0][1]) < 1e-15


def test_mirrored_mesh_mirrors_geometry():
    # reversing the xi index and reflecting x -> -x keeps the handedness and must
    # turn g_xi(q) into -P g_xi(q') with P = diag(-1, 1): D_{+1} and D_{-1} swap roles
    mesh = W.periodic_sine_mesh(16, 0.02)
    X = mesh["x"][::-1].copy()
    X[..., 0] *= -1.0
    mir = W._mesh(2, mesh["n"], X, (0, 0), shift=[[16, 0], [0, 16]])
    P = np.diag([-1.0, 1.0, 1.0])
    for qi in [(0, 0, 0), (3, 7, 0), (15, 2, 0)]:
        a = cell_geometry(mesh, qi)
        b = cell_geometry(mir, (15 - qi[0], qi[1], 0))
        assert np.allclose(b["g_low"][0], -(P @ a["g_low"][0]), atol=1e-14)
        assert np.allclose(b["g_low"][1], P @ a["g_low"][1], atol=1e-14)
        assert abs(a["J"] - b["J"]) < 1e-14


def test_affine_mesh_closed_form():
    A = np.array([[1.2, 0.3, -0.1], [0.05, 0.85, 0.2], [0.1, -0.15, 1.05]])
    mesh = W.affine_mesh(A, (5, 4, 3))
    for qi in [(0, 0, 0), (4, 3, 2), (2, 1, 1)]:
        g = cell_geometry(mesh, qi)
        assert np.allclose(g["g_low"], A.T, atol=1e-14)
        assert abs(g["J"] - np.linalg.det(A)) < 1e-14
        assert np.allclose(g["ginv"], np.linalg.inv(A.T @ A), atol=1e-13)
        # Theta vanishes on a uniform (affine) lattice (text after Eq. 11)
        assert np.abs(g["theta"]).max() < 1e-14


def _polar(nr=12, nth=12, r0=20.0, dr=1.0, dth=0.05):
    return W.polar_periodic_mesh(nr, nth, r0, dr, dth), r0, dr, dth


def test_polar_mesh_exact_theta():
    """Closed form of Eqs. 1, 3, 5, 7, 11 on r = r0 + i dr, theta = j dtheta.

    g_r = dr rhat, g_theta = 2 r sin(dth/2) thetahat (chord length, beta = sec(dth/2)),
    and for a link reaching (r', theta + b dth):
      Theta^r_r = cos(b dth) - 1,          Theta^th_r = dr sin(b dth) / (2 r s)
      Theta^r_th = -2 r' s sin(b dth)/dr,  Theta^th_th = (r'/r) cos(b dth) - 1
    with s = sin(dth/2).
    """
    mesh, r0, dr, dth = _polar()
    c, w, T0 = lattice(9)
    s = math.sin(dth / 2)
    for (i, j) in [(3, 4), (5, 6), (8, 7)]:
        g = cell_geometry(mesh, (i, j, 0))
        r, th = r0 + i * dr, j * dth
        rh = np.array([math.cos(th), math.sin(th), 0])
        thh = np.array([-math.sin(th), math.cos(th), 0])
        assert np.allclose(g["g_low"][0], dr * rh, atol=1e-13)
        assert np.allclose(g["g_low"][1], 2 * r * s * thh, atol=1e-12)
        assert abs(g["J"] - dr * 2 * r * s) < 1e-12
        for a in range(9):
            ca, cb = c[a][0], c[a][1]
            rp = r + ca * dr
            b = cb
            exact = np.array([[math.cos(b * dth) - 1.0, -2 * rp * s * math.sin(b * dth) / dr],
                              [dr * math.sin(b * dth) / (2 * r * s), (rp / r) * math.cos(b * dth) - 1.0]])
            assert np.allclose(g["theta"][a][:2, :2], exact, atol=1e-12, rtol=1e-12), (a, g["theta"][a], exact)


def test_theta_tends_to_christoffel():
    """Eqs. 63-66: Theta^i_j(q +- c, q) -> +- c^k Gamma^i_jk under refinement.
    In index coordinates of the polar map: Gamma^th_{r th} = Gamma^th_{th r} = dr/r,
    Gamma^r_{th th} = -r dth^2/dr."""
    c, w, T0 = lattice(9)
    errs = []
    for ref in (1, 2, 4):
        r0 = 20.0
        dr = 1.0 / ref
        dth = 0.05 / ref
        mesh = W.polar_periodic_mesh(6, 6, r0, dr, dth)
        g = cell_geometry(mesh, (3, 3, 0))
        r = r0 + 3 * dr
        Gam = np.zeros((2, 2, 2))
        Gam[1, 0, 1] = Gam[1, 1, 0] = dr / r
        Gam[0, 1, 1] = -r * dth ** 2 / dr
        e = 0.0
        for a in range(1, 9):
            lim = np.einsum("k,ijk->ij", c[a][:2].astype(float), Gam)
            e = max(e, np.abs(g["theta"][a][:2, :2] - lim).max() / np.abs(lim).max())
        errs.append(e)
    assert errs[-1] < 0.1
    assert errs[0] / errs[1] > 1.8 and errs[1] / errs[2] > 1.8


def test_degenerate_mesh_is_rejected():
    mesh = W.periodic_sine_mesh(8, 0.0)
    X = mesh["x"].copy()
    X[4, 3, 0] = X[2, 3, 0]          # both xi-neighbours of (3, 3) coincide: D_1 = D_-1
    bad = W._mesh(2, (8, 8, 1), X, (0, 0), shift=[[8, 0], [0, 8]])
    with pytest.raises(OracleError) as e:
        cell_geometry(bad, (3, 3, 0))
    assert e.value.code == "EGEOM"
    # left-handed mesh: J < 0
    Xl = mesh["x"][:, ::-1].copy()
    left = W._mesh(2, (8, 8, 1), Xl, (0, 0), shift=[[8, 0], [0, -8]])
    with pytest.raises(OracleError) as e2:
        cell_geometry(left, (2, 2, 0))
    assert e2.value.code == "EGEOM"
