"""CPU reference of the warm-start U-Net (include/vlb_nn.h), written with plain
PyTorch CPU operations in FP64, for checking the CUDA forward and backward
passes. Shares nothing with the CUDA code but the published topology."""
import numpy as np


def unpack(params, shapes):
    import torch
    out, o = [], 0
    for co, ci, k in shapes:
        nw = co * ci * k * k
        w = torch.tensor(params[o:o + nw].astype(np.float64).reshape(co, ci, k, k), requires_grad=True)
        o += nw
        b = torch.tensor(params[o:o + co].astype(np.float64), requires_grad=True)
        o += co
        out.append((w, b))
    assert o == len(params)
    return out


def forward(x, layers):
    import torch
    import torch.nn.functional as F

    def c(h, i, relu=True):
        w, b = layers[i]
        y = F.conv2d(h, w, b, padding=w.shape[-1] // 2)
        return F.relu(y) if relu else y

    up = lambda h: F.interpolate(h, scale_factor=2, mode="nearest")  # noqa: E731
    e1 = c(x, 0)
    s1 = c(e1, 1)
    e2 = c(F.avg_pool2d(s1, 2), 2)
    s2 = c(e2, 3)
    e3 = c(F.avg_pool2d(s2, 2), 4)
    b = c(e3, 5)
    d2 = c(torch.cat([up(b), s2], 1), 6)
    t2 = c(d2, 7)
    d1 = c(torch.cat([up(t2), s1], 1), 8)
    t1 = c(d1, 9)
    return c(t1, 10, relu=False)


def flat_grads(layers):
    return np.concatenate([np.concatenate([w.grad.numpy().ravel(), b.grad.numpy().ravel()]) for w, b in layers])
