"""The schedule network's CUDA kernels (through the C ABI) against the FP64
oracle in oracle/mlp.py.

Bar (FP32 kernels against an FP64 definition): forward outputs within 1e-5
of max |o|; loss within 1e-5 relative; the gradient within 1e-4 relative
2-norm; the first Adam step moves a coordinate by -lr g / (|g| + eps) to
FP32 rounding.  Row counts span many warps and blocks with
ragged tails (1000 = 31 * 32 + 8 rows)."""
import numpy as np
import pytest

from oracle import mlp as M

from gpu_helpers import dev, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return require_gpu()


def _data(seed, B):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1.5, 1.5, (B, 12))
    Y = np.stack([rng.uniform(0, 1, B), rng.integers(0, 2, B).astype(float)], 1)
    mask = (rng.uniform(0, 1, B) < 0.7).astype(float)
    return X, Y, mask


def _theta(seed):
    th = M.init_params(seed).astype(np.float32)
    th[-2:] = [0.3, -0.2]
    return th


@pytest.mark.parametrize("B", [1, 7, 1000])
def test_forward_matches_oracle(env, B):
    torch, ei = env
    th = _theta(11)
    X, _, _ = _data(1, B)
    X32 = X.astype(np.float32)
    net = ei.Mlp()
    net.set_params(th)
    assert np.array_equal(net.get_params(), th)
    out = torch.empty((B, 2), dtype=torch.float32, device="cuda")
    net.forward(dev(torch, X32), out)
    torch.cuda.synchronize()
    ref = M.forward(th.astype(np.float64), X32.astype(np.float64))
    got = out.cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("seed", [0, 1])
def test_loss_and_gradient_match_oracle(env, seed):
    torch, ei = env
    th = _theta(20 + seed)
    X, Y, mask = _data(seed, 1000)
    X32, Y32, m32 = X.astype(np.float32), Y.astype(np.float32), mask.astype(np.float32)
    lam, kappa = 0.3, 4.0
    net = ei.Mlp()
    net.set_params(th)
    grad = torch.empty(ei.MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = net.loss_grad(dev(torch, X32), dev(torch, Y32), dev(torch, m32), grad, lam, kappa)
    lref, gref = M.loss_grad(th.astype(np.float64), X32.astype(np.float64),
                             Y32.astype(np.float64), m32.astype(np.float64), lam, kappa)
    g = grad.cpu().numpy().astype(np.float64)
    assert loss == pytest.approx(lref, rel=1e-5)
    assert np.linalg.norm(g - gref) <= 1e-4 * np.linalg.norm(gref)


def test_all_masked_rows_leave_only_the_classifier(env):
    """mask 0 everywhere: the regression term and its gradient vanish; the
    gradient of the first output's bias is exactly 0."""
    torch, ei = env
    th = _theta(5)
    X, Y, _ = _data(3, 300)
    net = ei.Mlp()
    net.set_params(th)
    grad = torch.empty(ei.MLP_PARAMS, dtype=torch.float32, device="cuda")
    z = np.zeros(300, dtype=np.float32)
    loss = net.loss_grad(dev(torch, X.astype(np.float32)), dev(torch, Y.astype(np.float32)),
                         dev(torch, z), grad, 0.5, 4.0)
    lref = M.loss(th.astype(np.float64), X.astype(np.float32).astype(np.float64),
                  Y.astype(np.float32).astype(np.float64), z.astype(np.float64), 0.5, 4.0)
    assert loss == pytest.approx(lref, rel=1e-5)
    assert grad.cpu().numpy()[-2] == 0.0


def test_first_adam_step(env):
    torch, ei = env
    th = _theta(7)
    X, Y, mask = _data(4, 500)
    X32, Y32, m32 = (a.astype(np.float32) for a in (X, Y, mask))
    net = ei.Mlp()
    net.set_params(th)
    lr = 1e-3
    net.train_step(dev(torch, X32), dev(torch, Y32), dev(torch, m32), lr)
    th1 = net.get_params().astype(np.float64)
    _, g = M.loss_grad(th.astype(np.float64), X32.astype(np.float64), Y32.astype(np.float64),
                       m32.astype(np.float64))
    # bias-corrected moments after one step are g and g^2: the step is
    # -lr g / (|g| + eps); coordinates whose gradient is tiny against the
    # largest are left out (FP32 rounding can flip their sign)
    sel = np.abs(g) > 1e-3 * np.abs(g).max()
    step = th1 - th.astype(np.float64)
    np.testing.assert_allclose(step[sel], -lr * g[sel] / (np.abs(g[sel]) + 1e-8), rtol=2e-3,
                               atol=5e-7)


def test_training_reduces_loss(env):
    """300 Adam steps on a smooth target cut the loss by an order of magnitude."""
    torch, ei = env
    rng = np.random.default_rng(9)
    X = rng.uniform(-1, 1, (2048, 12)).astype(np.float32)
    Y = np.stack([0.5 + 0.3 * np.tanh(X[:, 0] - X[:, 3]), (X[:, 1] > 0)], 1).astype(np.float32)
    mask = np.ones(2048, dtype=np.float32)
    net = ei.Mlp()
    net.set_params(M.init_params(3).astype(np.float32))
    Xd, Yd, md = dev(torch, X), dev(torch, Y), dev(torch, mask)
    l0 = net.train_step(Xd, Yd, md, 3e-3)
    for _ in range(300):
        net.train_step(Xd, Yd, md, 3e-3, want_loss=False)
    l1 = net.train_step(Xd, Yd, md, 3e-3)
    assert l1 < 0.1 * l0
    # the trained parameters reproduce the oracle's loss
    lref = M.loss(net.get_params().astype(np.float64), X.astype(np.float64),
                  Y.astype(np.float64), mask.astype(np.float64))
    grad = torch.empty(ei.MLP_PARAMS, dtype=torch.float32, device="cuda")
    assert net.loss_grad(Xd, Yd, md, grad) == pytest.approx(lref, rel=1e-4)
