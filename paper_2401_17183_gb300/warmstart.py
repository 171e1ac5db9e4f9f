"""The learned warm start: steady solutions from the solver, the network's
features and targets, training, and the time-to-steady comparison.

Geometry family (2D, D2Q9, FP32): bumped channels of H x W = 32 x 64 cells
(channel2d_mesh): wall-normal tanh stretching in [0.3, 0.8], a lower-wall bump
of 0 to 0.15 of the half height, and a body force along the periodic axis of
5e-6 to 3e-5 (centre-line Reynolds number about 2 to 12 at tau = 0.8). Every
value is drawn from the counter-based generator of the workloads module.

Steady state: the residual r = ||u~^n - u~^(n-100)||_2 / (100 ||u~^n||_2),
checked every 100 steps, below tol (1e-6).

Network input (8 channels per cell): node position (x / W, y / h), J - 1,
g^11 - 1, g^12, g^22 - 1, the body force scaled to [0, 1] and the wall-normal
index position; output (3 channels): rho - 1 and the Euclidean u~, each
divided by a scale fixed from the training set. All of the network's
arithmetic runs in the library's CUDA kernels (nn.Net); this module marshals
arrays and drives the loops.
"""
import time

import numpy as np

from . import nn as _nn
from . import vlb
from . import workloads as W

H, WD = 32, 64
TAU = 0.8
G_LO, G_HI = 5e-6, 3e-5
CHECK = 100


def family(seed, n):
    """n seeded members of the geometry family: (stretch, bump, G)."""
    u = W.uniform(seed, n, 3)
    return [(0.3 + 0.5 * u[k, 0], 0.15 * u[k, 1], G_LO + (G_HI - G_LO) * u[k, 2]) for k in range(n)]


def make_member(spec):
    stretch, bump, G = spec
    mesh = W.channel2d_mesh(H, WD, stretch=stretch, bump=bump)
    return mesh, W.params(TAU, body_force=(0.0, G, 0.0))


def features(mesh, G, vmesh):
    """(8, H, W) float32 network input for one member."""
    x = W.node_positions(mesh).reshape(H, WD, 2)
    geo = vmesh.geometry()
    J, ginv = geo["J"], geo["ginv"]
    h = 0.5 * H
    f = np.empty((8, H, WD), dtype=np.float32)
    f[0] = x[..., 1] / WD
    f[1] = x[..., 0] / h
    f[2] = (J - 1.0).reshape(H, WD)
    f[3] = (ginv[:, 0, 0] - 1.0).reshape(H, WD)
    f[4] = ginv[:, 0, 1].reshape(H, WD)
    f[5] = (ginv[:, 1, 1] - 1.0).reshape(H, WD)
    f[6] = (G - G_LO) / (G_HI - G_LO)
    f[7] = ((np.arange(H) + 0.5) / H)[:, None]
    return f


def fields(sim):
    m = sim.moments()
    return m["rho"].reshape(H, WD), m["u_tilde"].reshape(H, WD, 2)


def residual(prev, cur):
    return float(np.linalg.norm(cur - prev) / (CHECK * max(np.linalg.norm(cur), 1e-300)))


def run_to_steady(sims, tol=1e-6, max_steps=30000):
    """Advance the members together (one batch launch per step) until each one's
    residual is below tol; returns the steps each needed (max_steps + CHECK
    for one that did not get there) and the wall time."""
    t0 = time.perf_counter()
    batch = vlb.Batch(sims)
    prev = [fields(s)[1] for s in sims]
    steps = np.full(len(sims), -1, dtype=np.int64)
    done = 0
    while done < max_steps and (steps < 0).any():
        batch.step(CHECK)
        done += CHECK
        for k, s in enumerate(sims):
            if steps[k] >= 0:
                continue
            cur = fields(s)[1]
            if residual(prev[k], cur) < tol:
                steps[k] = done
            prev[k] = cur
    batch.close()
    steps[steps < 0] = max_steps + CHECK
    return steps, time.perf_counter() - t0


def make_sims(specs, init=None):
    """Simulations of the members, started at rest or from init[k] = (rho, u)."""
    out = []
    for k, spec in enumerate(specs):
        mesh, prm = make_member(spec)
        vm = vlb.Mesh(mesh)
        if init is None:
            rho, u = W.rest_fields(mesh)
        else:
            rho = np.ascontiguousarray(init[k][0].reshape(-1), dtype=np.float64)
            u = np.ascontiguousarray(init[k][1].reshape(-1, 2), dtype=np.float64)
        out.append((mesh, vm, vlb.Sim(vm, prm, rho, u, precision=vlb.VLB_F32)))
    return out


def dataset(specs, steady_steps=12000, tol=1e-6):
    """Inputs and steady targets for the members: every member runs
    steady_steps steps from rest (one batch), then 100 more to check the
    residual; members above tol are dropped."""
    members = make_sims(specs)
    sims = [m[2] for m in members]
    batch = vlb.Batch(sims)
    batch.step(steady_steps)
    before = [fields(s) for s in sims]
    batch.step(CHECK)
    X, Y, keep = [], [], []
    for k, (mesh, vm, s) in enumerate(members):
        rho, ut = fields(s)
        if residual(before[k][1], ut) >= tol:
            continue
        X.append(features(mesh, specs[k][2], vm))
        Y.append(np.stack([rho - 1.0, ut[..., 0], ut[..., 1]]).astype(np.float32))
        keep.append(k)
    batch.close()
    return np.stack(X), np.stack(Y), keep


class WarmStart:
    """The trained network with its output scales."""

    def __init__(self, width=64, batch=32, storage=_nn.VLB_NN_BF16, seed=7):
        self.net = _nn.Net(8, 3, width, H, WD, batch, storage=storage, seed=seed)
        self.batch = batch
        self.scale = np.ones(3, dtype=np.float32)

    def train(self, X, Y, iters, lr=1e-3, seed=11, log=None):
        import torch
        self.scale = np.maximum(Y.std(axis=(0, 2, 3)), 1e-12).astype(np.float32)
        Ys = Y / self.scale[None, :, None, None]
        dX = torch.from_numpy(X).cuda()
        dY = torch.from_numpy(Ys).cuda()
        B = self.batch
        out = torch.zeros((B, 3, H, WD), dtype=torch.float32, device="cuda")
        dout = torch.zeros_like(out)
        rng = np.random.default_rng(seed)
        losses = []
        t0 = time.perf_counter()
        for it in range(1, iters + 1):
            idx = torch.from_numpy(rng.choice(len(X), B, replace=False)).cuda()
            xb = dX.index_select(0, idx).contiguous()
            yb = dY.index_select(0, idx).contiguous()
            self.net.forward(xb.data_ptr(), out.data_ptr(), B)
            losses.append(self.net.mse(out.data_ptr(), yb.data_ptr(), dout.data_ptr(), B))
            self.net.backward(dout.data_ptr(), B)
            self.net.adam(lr * (0.1 ** (it / iters)), it)
            if log and (it % 200 == 0 or it == iters):
                log("iter %d loss %.3e" % (it, losses[-1]))
        return losses, time.perf_counter() - t0

    def predict(self, X):
        """Steady (rho, u~) estimates for inputs X (n, 8, H, W)."""
        import torch
        outs = []
        B = self.batch
        for i in range(0, len(X), B):
            xb = np.zeros((B, 8, H, WD), dtype=np.float32)
            nb = min(B, len(X) - i)
            xb[:nb] = X[i:i + nb]
            dx = torch.from_numpy(xb).cuda()
            dy = torch.zeros((B, 3, H, WD), dtype=torch.float32, device="cuda")
            self.net.forward(dx.data_ptr(), dy.data_ptr(), B)
            outs.append(dy.cpu().numpy()[:nb])
        Y = np.concatenate(outs) * self.scale[None, :, None, None]
        return [(1.0 + y[0], np.stack([y[1], y[2]], -1)) for y in Y]
