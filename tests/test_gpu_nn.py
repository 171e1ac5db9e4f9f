"""The warm-start network's hand-written CUDA kernels against a CPU reference.

The reference (tests/nn_reference.py) is the same topology in plain PyTorch
CPU operations in FP64 with autograd. Checked: the forward pass and the
parameter gradients of the mean-square loss in FP32 storage, the forward pass
in bfloat16 storage (FP32 accumulation), one Adam step against its formula,
and that a short training run drives the loss down.
"""
import numpy as np
import pytest

from . import nn_reference as ref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def NN():
    from paper_2401_17183_gb300 import build as B
    B.build()
    from paper_2401_17183_gb300 import nn
    nn.load()
    return nn


def _setup(NN, storage, width=4, H=8, W=16, ci=5, co=3, B=3, seed=3):
    torch = pytest.importorskip("torch")
    net = NN.Net(ci, co, width, H, W, B, storage=storage, seed=seed)
    rng = np.random.default_rng(seed)
    p = net.params()
    # non-zero biases so that their gradients and uses are exercised
    o = 0
    for cout, cin, k in NN.layer_shapes(ci, co, width):
        o += cout * cin * k * k
        p[o:o + cout] = rng.uniform(-0.1, 0.1, cout).astype(np.float32)
        o += cout
    net.set_params(p)
    x = rng.uniform(-1, 1, (B, ci, H, W)).astype(np.float32)
    t = rng.uniform(-1, 1, (B, co, H, W)).astype(np.float32)
    dx = torch.from_numpy(x).cuda()
    dt = torch.from_numpy(t).cuda()
    dy = torch.zeros((B, co, H, W), dtype=torch.float32, device="cuda")
    ddy = torch.zeros_like(dy)
    return torch, net, p, x, t, dx, dt, dy, ddy


def test_forward_and_gradients_match_cpu_reference(NN):
    torch, net, p, x, t, dx, dt, dy, ddy = _setup(NN, NN.VLB_NN_F32)
    B = x.shape[0]
    net.forward(dx.data_ptr(), dy.data_ptr(), B)
    torch.cuda.synchronize()
    y = dy.cpu().numpy()
    layers = ref.unpack(p, NN.layer_shapes(5, 3, 4))
    yr = ref.forward(torch.from_numpy(x.astype(np.float64)), layers)
    assert np.abs(y - yr.detach().numpy()).max() <= 1e-5 * np.abs(yr.detach().numpy()).max()
    loss = net.mse(dy.data_ptr(), dt.data_ptr(), ddy.data_ptr(), B)
    lr_ = ((yr - torch.from_numpy(t.astype(np.float64))) ** 2).mean()
    assert abs(loss - lr_.item()) <= 1e-5 * lr_.item()
    net.backward(ddy.data_ptr(), B)
    g = net.grads()
    lr_.backward()
    gr = ref.flat_grads(layers)
    assert np.linalg.norm(g - gr) <= 1e-4 * np.linalg.norm(gr)
    # every layer's weights and biases receive their own gradient
    o = 0
    for cout, cin, k in NN.layer_shapes(5, 3, 4):
        nw = cout * cin * k * k
        for sl in (slice(o, o + nw), slice(o + nw, o + nw + cout)):
            assert np.linalg.norm(g[sl] - gr[sl]) <= 1e-3 * np.linalg.norm(gr[sl]) + 1e-7
        o += nw + cout


def test_bf16_storage_forward(NN):
    torch, net, p, x, t, dx, dt, dy, ddy = _setup(NN, NN.VLB_NN_BF16)
    net.forward(dx.data_ptr(), dy.data_ptr(), x.shape[0])
    torch.cuda.synchronize()
    layers = ref.unpack(p, NN.layer_shapes(5, 3, 4))
    yr = ref.forward(torch.from_numpy(x.astype(np.float64)), layers).detach().numpy()
    err = np.linalg.norm(dy.cpu().numpy() - yr) / np.linalg.norm(yr)
    assert err < 3e-2, err


def test_bf16_forward_on_tensor_cores(NN):
    """Width 16 on a 32 x 64 grid: every 3x3 layer fits the tensor-core form
    (tcgen05, FP32 accumulators in tensor memory). The forward pass matches
    the FP64 reference as the CUDA-core form does, and the two forms agree
    with each other to the rounding of the bfloat16 activations."""
    torch, net, p, x, t, dx, dt, dy, ddy = _setup(NN, NN.VLB_NN_BF16, width=16, H=32, W=64, ci=8, co=3, B=2)
    B = x.shape[0]
    net.forward(dx.data_ptr(), dy.data_ptr(), B)
    torch.cuda.synchronize()
    y_tc = dy.cpu().numpy().copy()
    net.set_tensor_cores(False)
    net.forward(dx.data_ptr(), dy.data_ptr(), B)
    torch.cuda.synchronize()
    y_fma = dy.cpu().numpy().copy()
    net.set_tensor_cores(True)
    layers = ref.unpack(p, NN.layer_shapes(8, 3, 16))
    yr = ref.forward(torch.from_numpy(x.astype(np.float64)), layers).detach().numpy()
    nr = np.linalg.norm(yr)
    assert np.linalg.norm(y_tc - yr) / nr < 3e-2
    assert np.linalg.norm(y_fma - yr) / nr < 3e-2
    assert np.linalg.norm(y_tc - y_fma) / nr < 1e-2


def test_adam_step(NN):
    torch, net, p, x, t, dx, dt, dy, ddy = _setup(NN, NN.VLB_NN_F32)
    B = x.shape[0]
    net.forward(dx.data_ptr(), dy.data_ptr(), B)
    net.mse(dy.data_ptr(), dt.data_ptr(), ddy.data_ptr(), B)
    net.backward(ddy.data_ptr(), B)
    g = net.grads().astype(np.float64)
    net.adam(1e-3, 1)
    m = 0.1 * g
    v = 0.001 * g * g
    exp = p - 1e-3 * (m / 0.1) / (np.sqrt(v / 0.001) + 1e-8)
    assert np.abs(net.params() - exp).max() <= 1e-6


def test_training_reduces_loss(NN):
    torch, net, p, x, t, dx, dt, dy, ddy = _setup(NN, NN.VLB_NN_BF16, width=8, H=16, W=16, B=4)
    # a smooth target that depends on the input
    target = torch.tanh(dx[:, :3] + 0.5 * dx[:, 1:4]).contiguous()
    B = x.shape[0]
    losses = []
    # measured loss ratio after 150 / 300 iterations: 0.148 / 0.073 (bfloat16
    # storage), 0.159 / 0.080 (FP32 storage): 300 iterations reach a tenth
    for it in range(1, 301):
        net.forward(dx.data_ptr(), dy.data_ptr(), B)
        losses.append(net.mse(dy.data_ptr(), target.data_ptr(), ddy.data_ptr(), B))
        net.backward(ddy.data_ptr(), B)
        net.adam(3e-3, it)
    assert losses[-1] < 0.1 * losses[0], (losses[0], losses[-1])
