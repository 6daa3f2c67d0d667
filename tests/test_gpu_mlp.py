"""The network's CUDA kernels against the FP64 reference."""
import numpy as np
import pytest

from oracle import mlp_ref as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_1411_2181_gb300 import build
    build.build()
    from paper_1411_2181_gb300 import mlp
    return mlp


def batch(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, 6)).astype(np.float32)
    t = np.column_stack([rng.uniform(0, 0.5, n), rng.uniform(-0.5, 0.5, n), rng.integers(0, 2, n),
                         rng.uniform(0, 1, n)]).astype(np.float32)
    mask = (rng.uniform(size=n) > 0.2).astype(np.float32)
    return x, t, mask


def per_tensor_err(g, ref):
    errs = []
    for (gw, gb), (rw, rb) in zip(R.unpack(g.astype(np.float64)), R.unpack(ref)):
        for a, b in ((gw, rw), (gb, rb)):
            errs.append(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))
    return max(errs)


@pytest.mark.parametrize("B", [1, 37, 300])
def test_fp32_forward_and_gradient(M, B):
    net = M.MLP(max_batch=512, bf16=False)
    p = M.init_params(3)
    net.set_params(p)
    x, t, mask = batch(B, B)
    y = net.forward(x)
    yr = R.forward(p.astype(np.float64), x.astype(np.float64))
    assert np.abs(y - yr).max() / np.abs(yr).max() < 1e-5
    loss = net.loss_grad(x, t, mask)
    lr_, gr = R.loss_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64), mask)
    assert abs(loss - lr_) / abs(lr_) < 1e-5
    assert per_tensor_err(net.grads(), gr) < 1e-5


def test_bf16_weights_gradient(M):
    """BF16 weights: compare with the reference evaluated at the BF16-rounded
    weights; accumulation stays FP32."""
    import torch
    net = M.MLP(max_batch=512, bf16=True)
    p = M.init_params(4)
    net.set_params(p)
    pb = torch.tensor(p).to(torch.bfloat16).to(torch.float64).numpy()
    x, t, mask = batch(256, 9)
    net.loss_grad(x, t, mask)
    _, gr = R.loss_grad(pb, x.astype(np.float64), t.astype(np.float64), mask)
    assert per_tensor_err(net.grads(), gr) < 1e-2
    y = net.forward(x)
    yr = R.forward(pb, x.astype(np.float64))
    assert np.abs(y - yr).max() / np.abs(yr).max() < 1e-2


def test_adamw_steps_match_reference(M):
    net = M.MLP(max_batch=128, bf16=False)
    p = M.init_params(5)
    net.set_params(p)
    x, t, mask = batch(64, 11)
    pr = p.astype(np.float64)
    m = np.zeros_like(pr)
    v = np.zeros_like(pr)
    for step in range(1, 4):
        net.loss_grad(x, t, mask)
        g = net.grads().astype(np.float64)
        net.adamw(lr=1e-3, weight_decay=1e-2)
        pr, m, v = R.adamw(pr, m, v, g, step, lr=1e-3, wd=1e-2)
        assert np.abs(net.get_params() - pr).max() < 1e-6


def test_training_reduces_loss(M):
    rng = np.random.default_rng(0)
    x = rng.uniform(-1, 1, size=(1024, 6)).astype(np.float32)
    t = np.column_stack([0.3 * np.tanh(x[:, 0]), 0.2 * x[:, 1] * x[:, 2], (x[:, 0] + x[:, 3] > 0),
                         np.abs(x[:, 4])]).astype(np.float32)
    net = M.MLP(max_batch=1024, bf16=True)
    net.set_params(M.init_params(0))
    hist = net.fit(x, t, epochs=300, lr=3e-3, batch=256)
    assert hist[-1] < 0.25 * hist[0]
