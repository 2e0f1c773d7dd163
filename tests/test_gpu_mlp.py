"""Emulator network kernels against the FP64 oracle (oracle/mlp.py).

FP32 mode: forward, backward and Adam within 1e-5 (relative to the largest
value) of FP64. BF16 mode: against the oracle with the same bfloat16 rounding
of weights and activations applied, within 1e-2 (different FP32 accumulation
order can move a value across a bfloat16 rounding boundary)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import mlp as om  # noqa: E402
from paper_1807_04215_gb300 import gridspt as g  # noqa: E402
from tests import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def _setup(bf16, B=70, H=128, O=160, seed=0):
    net = g.MLP(3, H, O, bf16=bf16, seed=seed)
    r = inputs.rng(seed + 1)
    x = r.standard_normal((B, 3))
    t = r.standard_normal((B, O))
    mask = (r.random((B, O)) > 0.1).astype(float)
    dev = lambda a: torch.from_numpy(a.astype(np.float32)).cuda()  # noqa: E731
    return net, x, t, mask, dev


@pytest.mark.parametrize("bf16", [False, True])
def test_forward_backward_match_oracle(bf16):
    net, x, t, mask, dev = _setup(bf16)
    B = x.shape[0]
    theta = net.master.double().cpu().numpy()
    rnd = om.bf16_round if bf16 else om.ident
    xr = x.astype(np.float32).astype(np.float64)
    y_ref, acts = om.forward(xr, theta, net.H, net.O, rnd)
    act = torch.empty(B, 4 * net.H, dtype=torch.float32, device="cuda")
    y = net.forward(dev(x), act=act).double().cpu().numpy()
    tol = 1e-2 if bf16 else 1e-5
    assert np.abs(y - y_ref).max() <= tol * np.abs(y_ref).max()
    L, dy_ref = om.masked_mse(y_ref, t.astype(np.float32), mask)
    dy = torch.empty(B, net.O, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    net.mse(net.forward(dev(x), act=act), dev(t), dev(mask), dy, loss)
    assert abs(loss.item() - L) <= tol * L
    ws = torch.empty(net.ws_bytes(B), dtype=torch.uint8, device="cuda")
    grad = net.backward(dev(x), act, dev(dy_ref), ws).double().cpu().numpy()
    g_ref = om.backward(xr, theta, net.H, net.O, acts, dy_ref, rnd)
    assert np.abs(grad - g_ref).max() <= tol * np.abs(g_ref).max()


def test_backward_is_bitwise_repeatable():
    net, x, t, mask, dev = _setup(False, B=100)
    act = torch.empty(100, 4 * net.H, dtype=torch.float32, device="cuda")
    y = net.forward(dev(x), act=act)
    dy = dev(t)
    ws = torch.empty(net.ws_bytes(100), dtype=torch.uint8, device="cuda")
    a = net.backward(dev(x), act, dy, ws).clone()
    b = net.backward(dev(x), act, dy, ws).clone()
    assert torch.equal(a, b)


def test_adam_matches_oracle_over_steps():
    net, x, t, mask, dev = _setup(False, B=40, H=16, O=8)
    theta = net.master.double().cpu().numpy()
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    r = inputs.rng(9)
    for step in range(1, 4):
        gr = r.standard_normal(theta.size)
        net.grad.copy_(torch.from_numpy(gr.astype(np.float32)))
        net.adam(1e-2)
        theta, m, v = om.adam_step(theta, gr.astype(np.float32).astype(np.float64), m, v, step, 1e-2)
    got = net.master.double().cpu().numpy()
    assert np.abs(got - theta).max() <= 1e-5 * np.abs(theta).max()
    assert int(net.step.item()) == 3


def test_training_reduces_loss():
    net, x, t, mask, dev = _setup(True, B=64, H=32, O=10)
    xs = torch.from_numpy(np.linspace(-1, 1, 64 * 3).reshape(64, 3).astype(np.float32)).cuda()
    ts = torch.sin(3 * xs[:, :1]) * torch.ones(1, 10, device="cuda")
    ms = torch.ones(64, 10, device="cuda")
    act = torch.empty(64, 4 * 32, dtype=torch.float32, device="cuda")
    dy = torch.empty(64, 10, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    ws = torch.empty(net.ws_bytes(64), dtype=torch.uint8, device="cuda")
    losses = []
    for it in range(300):
        y = net.forward(xs, act=act)
        net.mse(y, ts, ms, dy, loss)
        net.backward(xs, act, dy, ws)
        net.adam(3e-3)
        if it % 50 == 0:
            losses.append(loss.item())
    assert losses[-1] < 0.2 * losses[0]
