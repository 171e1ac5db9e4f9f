"""The rearranged force map used by the CUDA collision, checked on CPU.

The step kernel does not evaluate Eq. 27 direction by direction. It uses a
reduced form, Phi = J F:

    Phi_new = Pb' - 1/2 { m [PE : U~U~ + PO2 : (U~^k)^2 U~^l + LO U~] + TL Phi },

where the coefficient blocks PE, PO2, LO, TL (and CE, PO1 inside Pb') depend
only on the cell geometry and tau. That form follows from Eqs. 27, 30, 31 and
33 by linear algebra on the pair sums over directions. Here numpy re-derives
the blocks from the geometry (independently of the CUDA sources) and checks

  - that the reduced map equals the direct evaluation of Eqs. 27/30/31/33 for
    arbitrary Phi, populations and geometry (D2Q9 and D3Q19);
  - that the chord iteration with H = (I + LO/4 + TL/2)^-1 converges to the
    oracle's F;
  - that the chord step the kernel takes, Phi <- H (Pc - 1/2 m Q(U~)) with
    Pc = Pb' - 1/2 m LO U and Q = PE : U~U~ + PO2 : (U~^k)^2 U~^l (the linear
    part of the map cancels against H exactly), equals Phi + H (map(Phi) - Phi)
    computed from the direct evaluation, and reaches the oracle's F.

A wrong sign, a dropped term or a transposed index in the derivation fails
the first check by many orders of magnitude above round-off.
"""
import numpy as np
import pytest

from oracle import cell_geometry, collide, equilibrium, lattice
from paper_2401_17183_gb300 import workloads as W

T0 = 1.0 / 3.0


def _blocks(q, g, tau):
    """Coefficient blocks of the reduced map from one cell's geometry."""
    D = 2 if q == 9 else 3
    c, w, _ = lattice(q)
    c = c[:, :D].astype(float)
    K = np.einsum('aij,aj->ai', g['theta'][:, :D, :D], c)  # K^i_a = sum_j c^j_a Theta^i_j
    gd = g['ginv'][:D, :D] - np.eye(D)
    opp = [int(np.where((c == -c[a]).all(1))[0][0]) for a in range(q)]
    P = [a for a in range(1, q) if a < opp[a]]
    M = np.array([K[p] + K[opp[p]] for p in P])
    Dk = np.array([K[p] - K[opp[p]] for p in P])
    cp = np.array([c[p] for p in P])
    wp = np.array([w[p] for p in P])
    itau = 1.0 / tau
    cpi = -(1.0 - 0.5 * itau)
    ccI = 3 * np.einsum('pk,pl->pkl', cp, cp) - np.eye(D)[None]
    R = np.einsum('p,pi,pkl->ikl', wp, M, ccI)
    Ao = wp[:, None] * (itau * Dk + 3 * cpi * np.einsum('pk,ikl,pl->pi', cp, R, M))
    PE = 1.5 * itau * R
    PO1 = 3 * np.einsum('pi,pl->il', Ao, cp)
    PO2 = np.zeros((D, D, D))
    for k in range(D):
        for l in range(D):
            if k != l:
                PO2[:, k, l] = 4.5 * np.einsum('pi,p->i', Ao, cp[:, l] * (3 * cp[:, k] ** 2 - 1))
    TT = 3 * np.einsum('p,pi,pj->ij', wp, Dk, cp)
    LO = np.zeros((D, D))
    LD = np.zeros((D, D))
    for j in range(D):
        for k in range(D):
            if k != j:
                LO[:, j] += T0 * (PO2[:, k, j] * gd[k, k] + 2 * PO2[:, j, k] * gd[j, k])
                LD[:, j] += T0 * PO2[:, k, j]
    TL = TT + 0.5 * LD
    CE = T0 * np.einsum('ikl,kl->i', PE, gd)
    return dict(D=D, c=c, w=w, K=K, opp=opp, PE=PE, PO1=PO1, PO2=PO2, LO=LO, TL=TL, CE=CE)


def _maps(q, g, tau, N, G):
    b = _blocks(q, g, tau)
    D, c, w, K, opp = b['D'], b['c'], b['w'], b['K'], b['opp']
    J = g['J']
    itau = 1.0 / tau
    m = N.sum()
    rho = m / J
    U = (c.T @ N) / m
    L = -K[opp]
    # everything that does not change with Phi
    Pb = (m * G + 0.5 * L.T @ N - 0.5 * (1 - itau) * (K.T @ N) - 0.5 * itau * m * (K.T @ w)
          - 0.5 * m * (b['CE'] + b['PO1'] @ U))

    def reduced(Phi):
        Ut = U + Phi / (2 * m)
        cub = sum(b['PO2'][:, k, l] * Ut[k] ** 2 * Ut[l]
                  for k in range(D) for l in range(D) if k != l)
        a = np.einsum('ikl,k,l->i', b['PE'], Ut, Ut) + cub + b['LO'] @ Ut
        return Pb - 0.5 * (m * a + b['TL'] @ Phi)

    def direct(Phi):
        F = Phi / J
        Ut = U + F / (2 * rho)
        feq = equilibrium(q, rho, U, Ut, g['ginv'])[:q]
        dP = -0.5 * (1 - 0.5 * itau) * np.einsum('ai,aj,a->ij', c, K - L, feq)
        dN = w * J * (3 * (c @ F) + 3 * (3 * np.einsum('ai,ij,aj->a', c, dP, c) - np.trace(dP)))
        Np = N - (N - J * feq) * itau + dN
        return m * G - 0.5 * K.T @ Np + 0.5 * L.T @ N

    H = np.linalg.inv(np.eye(D) + 0.25 * b['LO'] + 0.5 * b['TL'])

    def folded(Phi):
        """One chord step in the form the CUDA collision evaluates it."""
        Ut = U + Phi / (2 * m)
        cub = sum(b['PO2'][:, k, l] * Ut[k] ** 2 * Ut[l]
                  for k in range(D) for l in range(D) if k != l)
        Qn = np.einsum('ikl,k,l->i', b['PE'], Ut, Ut) + cub
        Pc = Pb - 0.5 * m * (b['LO'] @ U)
        return H @ (Pc - 0.5 * m * Qn)

    reduced.folded = folded
    return reduced, direct, H


def _cases():
    chan = W.channel_mesh(16, 12, 8, stretch=0.7, bump=0.05)
    sine = W.periodic_sine_mesh(32, 0.02)
    polar = W.polar_mesh(16, 3, 30.0, 36.0, dtheta=1.0 / 33)
    return [(19, chan, (3, 0, 2)), (19, chan, (5, 5, 1)), (19, chan, (7, 11, 4)),
            (9, sine, (3, 7, 0)), (9, sine, (20, 11, 0)), (9, polar, (0, 1, 0)), (9, polar, (15, 2, 0))]


@pytest.mark.parametrize("case", range(7))
@pytest.mark.parametrize("tau", [0.6, 0.8, 1.3])
def test_reduced_map_equals_direct_evaluation(case, tau):
    q, mesh, qi = _cases()[case]
    D = 2 if q == 9 else 3
    rng = np.random.default_rng(100 + case)
    G = 1e-4 * rng.uniform(-1, 1, 3)
    prm = W.params(tau, body_force=tuple(G))
    g = cell_geometry(mesh, qi, prm)
    U0 = 0.05 * rng.uniform(-1, 1, D)
    N = g['J'] * equilibrium(q, 1.0, U0, U0, g['ginv'])[:q] * (1 + 0.05 * rng.uniform(-1, 1, q))
    reduced, direct, _ = _maps(q, g, tau, N, g['G'][:D])
    for _ in range(4):
        Phi = 0.05 * rng.uniform(-1, 1, D)
        a, b = reduced(Phi), direct(Phi)
        assert np.abs(a - b).max() <= 1e-14 * max(1.0, np.abs(b).max()), (a, b)


@pytest.mark.parametrize("case", range(7))
def test_chord_iteration_reaches_the_oracle_force(case):
    q, mesh, qi = _cases()[case]
    D = 2 if q == 9 else 3
    tau = 0.8
    rng = np.random.default_rng(7 + case)
    prm = W.params(tau, body_force=(1e-5, 0, 0), tol=1e-15, max_iter=500)
    g = cell_geometry(mesh, qi, prm)
    U0 = 0.03 * rng.uniform(-1, 1, D)
    N = g['J'] * equilibrium(q, 1.0, U0, U0, g['ginv'])[:q] * (1 + 0.02 * rng.uniform(-1, 1, q))
    ref = collide(q, g, prm, N)
    reduced, _, H = _maps(q, g, tau, N, g['G'][:D])
    Phi = np.zeros(D)
    for it in range(30):
        d = H @ (reduced(Phi) - Phi)
        Phi = Phi + d
        if np.abs(d).max() < 1e-16:
            break
    # the chord step removes the linear part exactly, so few steps are needed
    assert it < 12
    assert np.abs(Phi / g['J'] - ref['F'][:D]).max() <= 1e-13 * max(1e-3, np.abs(ref['F']).max())


@pytest.mark.parametrize("case", range(7))
@pytest.mark.parametrize("tau", [0.6, 0.8, 1.3])
def test_folded_chord_step_equals_chord_step_of_direct_map(case, tau):
    q, mesh, qi = _cases()[case]
    D = 2 if q == 9 else 3
    rng = np.random.default_rng(300 + case)
    G = 1e-4 * rng.uniform(-1, 1, 3)
    prm = W.params(tau, body_force=tuple(G))
    g = cell_geometry(mesh, qi, prm)
    U0 = 0.05 * rng.uniform(-1, 1, D)
    N = g['J'] * equilibrium(q, 1.0, U0, U0, g['ginv'])[:q] * (1 + 0.05 * rng.uniform(-1, 1, q))
    reduced, direct, H = _maps(q, g, tau, N, g['G'][:D])
    for _ in range(4):
        Phi = 0.05 * rng.uniform(-1, 1, D)
        chord = Phi + H @ (direct(Phi) - Phi)
        a = reduced.folded(Phi)
        assert np.abs(a - chord).max() <= 1e-14 * max(1.0, np.abs(chord).max()), (a, chord)


@pytest.mark.parametrize("case", range(7))
def test_folded_chord_iteration_reaches_the_oracle_force(case):
    q, mesh, qi = _cases()[case]
    D = 2 if q == 9 else 3
    tau = 0.8
    rng = np.random.default_rng(17 + case)
    prm = W.params(tau, body_force=(1e-5, 0, 0), tol=1e-15, max_iter=500)
    g = cell_geometry(mesh, qi, prm)
    U0 = 0.03 * rng.uniform(-1, 1, D)
    N = g['J'] * equilibrium(q, 1.0, U0, U0, g['ginv'])[:q] * (1 + 0.02 * rng.uniform(-1, 1, q))
    ref = collide(q, g, prm, N)
    reduced, _, _ = _maps(q, g, tau, N, g['G'][:D])
    Phi = np.zeros(D)
    for it in range(30):
        nxt = reduced.folded(Phi)
        d = nxt - Phi
        Phi = nxt
        if np.abs(d).max() < 1e-16:
            break
    assert it < 12
    assert np.abs(Phi / g['J'] - ref['F'][:D]).max() <= 1e-13 * max(1e-3, np.abs(ref['F']).max())
