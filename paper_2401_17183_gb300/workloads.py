"""Seeded synthetic inputs: meshes (node positions x(q)) and initial fields.

This module holds no arithmetic of the lattice Boltzmann method. It builds the
inputs the method starts from: the node coordinates of a structured mesh
(section 2.1 starts from a given mesh), its boundary kinds and periodic
transforms, and seeded initial density and velocity fields. Both the CUDA path
and the CPU oracle receive identical arrays from here.

A mesh is a plain dict:
  dim, q       2 and 9 (D2Q9) or 3 and 19 (D3Q19)
  n            (n0, n1, n2), n2 = 1 in 2D; axis 2 is the fastest in memory
  x            float64 array (n0, n1, n2, dim) of node positions
  bc           per axis 0 (periodic) or 1 (wall)
  shift, rot   periodic image across the +end of axis a is rot[a] @ x + shift[a]
               (rot[a] row-major 3x3; all zeros means identity)
  dx           representative spacing of Eq. 3
  wall_links   Theta on wall-crossing links: 0 zero, 1 from the ghost nodes
"""
import math

import numpy as np

PERIODIC = 0
WALL = 1

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(counter):
    """SplitMix64 output for each uint64 counter (Steele, Lea, Flood 2014)."""
    with np.errstate(over="ignore"):
        z = (np.asarray(counter, dtype=np.uint64) + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed, ncell, ncomp):
    """Counter-based uniform numbers in [0, 1), keyed by (seed, cell, component)."""
    cell = np.arange(ncell, dtype=np.uint64)[:, None]
    comp = np.arange(ncomp, dtype=np.uint64)[None, :]
    key = (np.uint64(seed) << np.uint64(40)) + cell * np.uint64(8) + comp
    z = splitmix64(key)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _mesh(dim, n, x, bc, shift=None, rot=None, dx=1.0, wall_links=0):
    n3 = (int(n[0]), int(n[1]), int(n[2]) if dim == 3 else 1)
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(n3 + (dim,)))
    sh = np.zeros((3, 3))
    if shift is not None:
        s = np.asarray(shift, dtype=np.float64)
        sh[:s.shape[0], :s.shape[1]] = s
    rt = np.zeros((3, 9))
    if rot is not None:
        r = np.asarray(rot, dtype=np.float64)
        rt[:r.shape[0], :r.shape[1]] = r
    bc3 = [int(b) for b in bc] + [PERIODIC] * (3 - len(bc))
    return {"dim": dim, "q": 9 if dim == 2 else 19, "n": n3, "x": x, "bc": tuple(bc3),
            "shift": sh, "rot": rt, "dx": float(dx), "wall_links": int(wall_links)}


def ncell(mesh):
    return int(mesh["n"][0] * mesh["n"][1] * mesh["n"][2])


def node_positions(mesh):
    """(ncell, dim) view of the node positions in cell order."""
    return mesh["x"].reshape(-1, mesh["dim"])


# --------------------------------------------------------------------------- meshes

def periodic_sine_mesh(L=64, amp_frac=0.1):
    """2D periodic mapped box: x = xi + A sin(2 pi eta / L), y = eta + A sin(2 pi xi / L)."""
    A = amp_frac * L
    xi, eta = np.meshgrid(np.arange(L, dtype=np.float64), np.arange(L, dtype=np.float64),
                          indexing="ij")
    x = xi + A * np.sin(2 * np.pi * eta / L)
    y = eta + A * np.sin(2 * np.pi * xi / L)
    X = np.stack([x, y], axis=-1)[:, :, None, :]
    return _mesh(2, (L, L, 1), X, (PERIODIC, PERIODIC), shift=[[L, 0], [0, L]])


def periodic_sine_mesh3d(L=16, amp_frac=0.01, q=19):
    """3D periodic mapped box: x = xi + A sin(2 pi eta / L), y = eta + A sin(2 pi
    zeta / L), z = zeta + A sin(2 pi xi / L); q selects the velocity set (19 or
    39, the 6th-order isotropic set)."""
    A = amp_frac * L
    g = np.arange(L, dtype=np.float64)
    xi, eta, zeta = np.meshgrid(g, g, g, indexing="ij")
    X = np.stack([xi + A * np.sin(2 * np.pi * eta / L), eta + A * np.sin(2 * np.pi * zeta / L),
                  zeta + A * np.sin(2 * np.pi * xi / L)], axis=-1)
    m = _mesh(3, (L, L, L), X, (PERIODIC, PERIODIC, PERIODIC), shift=[[L, 0, 0], [0, L, 0], [0, 0, L]])
    m["q"] = int(q)
    return m


def affine_mesh(A, n, b=None, dim=None):
    """Periodic affine mesh x = A q + b (every Theta vanishes)."""
    A = np.asarray(A, dtype=np.float64)
    dim = A.shape[0] if dim is None else dim
    n3 = tuple(n) + (1,) * (3 - len(n))
    grids = np.meshgrid(*[np.arange(n3[a], dtype=np.float64) for a in range(dim)], indexing="ij")
    Q = np.stack(grids, axis=-1)
    X = Q @ A.T
    if b is not None:
        X = X + np.asarray(b, dtype=np.float64)
    shift = [A[:, a] * n3[a] for a in range(dim)]
    return _mesh(dim, n3, X, [PERIODIC] * dim, shift=shift)


def channel_mesh(n0=256, n1=256, n2=256, stretch=2.5, bump=0.05, wall_links=0):
    """3D channel with a bumped lower wall, in lattice units.

    Axis 0 (xi) streamwise and periodic, axis 1 (eta) wall-normal with walls,
    axis 2 (zeta) spanwise and periodic (fastest in memory). The channel is
    2h = n1 high, n0 long and n2 wide, so mean spacings are one lattice unit.
    Wall-normal stretching y_s = h tanh(b (2 (eta + 1/2) / n1 - 1)) / tanh(b);
    the lower wall carries a bump of amplitude bump*h and wavelength n0/2,
    blended out linearly toward the upper wall. The mesh does not vary along
    zeta, so its geometry is one (xi, eta) plane repeated.
    """
    h = 0.5 * n1
    xi = np.arange(n0, dtype=np.float64)
    eta = np.arange(n1, dtype=np.float64)
    s = 2.0 * (eta + 0.5) / n1 - 1.0
    ys = h * np.tanh(stretch * s) / math.tanh(stretch) if stretch > 0 else h * s
    bl = bump * h * np.sin(2 * np.pi * xi / (0.5 * n0))
    y = ys[None, :] + bl[:, None] * (1.0 - ys[None, :] / h) / 2.0
    X = np.empty((n0, n1, n2, 3))
    X[..., 0] = xi[:, None, None]
    X[..., 1] = y[:, :, None]
    X[..., 2] = np.arange(n2, dtype=np.float64)[None, None, :]
    return _mesh(3, (n0, n1, n2), X, (PERIODIC, WALL, PERIODIC),
                 shift=[[n0, 0, 0], [0, 0, 0], [0, 0, n2]], wall_links=wall_links)


def channel_bump3d_mesh(n0=256, n1=256, n2=256, stretch=0.7, bump=0.05, wall_links=0):
    """3D channel as channel_mesh, but the lower-wall bump also varies along
    the spanwise axis, bump h sin(2 pi x / (n0/2)) cos(2 pi z / (n2/2)), so the
    geometry changes along every axis (no plane-invariant records)."""
    h = 0.5 * n1
    xi = np.arange(n0, dtype=np.float64)
    eta = np.arange(n1, dtype=np.float64)
    zeta = np.arange(n2, dtype=np.float64)
    s = 2.0 * (eta + 0.5) / n1 - 1.0
    ys = h * np.tanh(stretch * s) / math.tanh(stretch) if stretch > 0 else h * s
    bl = (bump * h * np.sin(2 * np.pi * xi / (0.5 * n0)))[:, None] * np.cos(2 * np.pi * zeta / (0.5 * n2))[None, :]
    X = np.empty((n0, n1, n2, 3))
    X[..., 0] = xi[:, None, None]
    X[..., 1] = ys[None, :, None] + bl[:, None, :] * (1.0 - ys[None, :, None] / h) / 2.0
    X[..., 2] = zeta[None, None, :]
    return _mesh(3, (n0, n1, n2), X, (PERIODIC, WALL, PERIODIC),
                 shift=[[n0, 0, 0], [0, 0, 0], [0, 0, n2]], wall_links=wall_links)


def channel2d_mesh(n0=32, n1=16, stretch=0.7, wall_links=0, bump=0.0):
    """2D channel: axis 0 wall-normal with walls and tanh stretching (as in
    channel_mesh), axis 1 streamwise, periodic and fastest in memory. Without
    a bump the geometry does not vary along axis 1; bump (a fraction of the
    half height h) raises the lower wall by bump h sin(2 pi x / n1), blended
    out linearly toward the upper wall."""
    h = 0.5 * n0
    s = 2.0 * (np.arange(n0, dtype=np.float64) + 0.5) / n0 - 1.0
    ys = h * np.tanh(stretch * s) / math.tanh(stretch) if stretch > 0 else h * s
    xs = np.arange(n1, dtype=np.float64)
    bl = bump * h * np.sin(2 * np.pi * xs / n1)
    X = np.empty((n0, n1, 2))
    X[..., 0] = ys[:, None] + bl[None, :] * (1.0 - ys[:, None] / h) / 2.0
    X[..., 1] = xs[None, :]
    return _mesh(2, (n0, n1, 1), X, (WALL, PERIODIC), shift=[[0, 0, 0], [0, n1, 0]],
                 wall_links=wall_links)


def polar_mesh(nr, ntheta, r_in, r_out, dtheta=None, wall_links=0):
    """2D annular sector: r_i = r_in + (i + 1/2) dr (walls at r_in, r_out),
    theta_j = j dtheta, periodic in theta through a rotation by ntheta dtheta."""
    dr = (r_out - r_in) / nr
    if dtheta is None:
        dtheta = 2 * np.pi / ntheta
    r = r_in + (np.arange(nr) + 0.5) * dr
    th = np.arange(ntheta) * dtheta
    R, T = np.meshgrid(r, th, indexing="ij")
    X = np.stack([R * np.cos(T), R * np.sin(T)], axis=-1)[:, :, None, :]
    ang = ntheta * dtheta
    rot = [[0] * 9, [math.cos(ang), -math.sin(ang), 0, math.sin(ang), math.cos(ang), 0, 0, 0, 1]]
    return _mesh(2, (nr, ntheta, 1), X, (WALL, PERIODIC), rot=rot, wall_links=wall_links)


def polar_periodic_mesh(nr, ntheta, r0, dr, dtheta):
    """Polar sector with a periodic radial axis treated only for geometry tests:
    nodes r_i = r0 + i dr, theta_j = j dtheta (no wrap is ever used in tests)."""
    r = r0 + np.arange(nr) * dr
    th = np.arange(ntheta) * dtheta
    R, T = np.meshgrid(r, th, indexing="ij")
    X = np.stack([R * np.cos(T), R * np.sin(T)], axis=-1)[:, :, None, :]
    return _mesh(2, (nr, ntheta, 1), X, (WALL, WALL))


# --------------------------------------------------------------------------- fields

def taylor_green_fields(mesh, L=64, amp=0.01, noise=1e-4, seed=1):
    """rho = 1; u = amp (sin kx cos ky, -cos kx sin ky) at the mapped node
    positions plus seeded uniform noise in [-noise, noise] per component."""
    X = node_positions(mesh)
    k = 2 * np.pi / L
    u = np.stack([amp * np.sin(k * X[:, 0]) * np.cos(k * X[:, 1]),
                  -amp * np.cos(k * X[:, 0]) * np.sin(k * X[:, 1])], axis=-1)
    u = u + noise * (2.0 * uniform(seed, X.shape[0], 2) - 1.0)
    return np.ones(X.shape[0]), np.ascontiguousarray(u)


def noise_fields(mesh, amp=0.01, seed=2, rho_amp=0.0):
    """rho = 1 (+ optional seeded noise); u uniform in [-amp, amp] per component."""
    nc = ncell(mesh)
    dim = mesh["dim"]
    r = uniform(seed, nc, dim + 1)
    u = amp * (2.0 * r[:, :dim] - 1.0)
    rho = 1.0 + rho_amp * (2.0 * r[:, dim] - 1.0)
    return np.ascontiguousarray(rho), np.ascontiguousarray(u)


def rest_fields(mesh):
    nc = ncell(mesh)
    return np.ones(nc), np.zeros((nc, mesh["dim"]))


def params(tau, body_force=(0.0, 0.0, 0.0), wall_u=None, wall_omega=None, max_iter=0,
           tol=0.0):
    return {"tau": float(tau), "body_force": tuple(float(v) for v in body_force) + (0.0,) * (3 - len(body_force)),
            "wall_u": None if wall_u is None else np.asarray(wall_u, dtype=np.float64),
            "wall_omega": None if wall_omega is None else np.asarray(wall_omega, dtype=np.float64),
            "max_iter": int(max_iter), "tol": float(tol)}


# --------------------------------------------------------------------------- instances

def precision_instance(n=64):
    """The storage-precision comparison instance: the channel family of the
    headline workload (tanh stretching 0.7, lower-wall bump 0.05 h) at n^3
    cells, tau = 0.8, body force 1e-5 streamwise (a channel flow of about
    0.01 after 1000 steps on top of the decaying noise), rho = 1 and seeded
    1% velocity noise. Returns (mesh, params, rho, u)."""
    mesh = channel_mesh(n, n, n, stretch=0.7, bump=0.05)
    prm = params(0.8, body_force=(1e-5, 0.0, 0.0))
    rho, u = noise_fields(mesh, amp=0.01, seed=3)
    return mesh, prm, rho, u
