"""A small fully connected network: forward pass, loss, backward pass, Adam.

ORACLE — test infrastructure only (see oracle/__init__.py).

The learned schedule maps features of a phi_1 call at a candidate substep
count to two numbers (the Leja degree the a posteriori estimate will need,
and whether it will be met within m_max); this module is the plain
definition of that network and of its training step, against which the CUDA
training and inference kernels are checked.  The paper itself has no network:
it fixes the substep count and degree by a conservative a priori rule
(Sec. III-C), which this replaces while the a posteriori estimate still
decides acceptance.

Definitions (standard, written out):

  * layers l = 0..L-1, h_0 = x, z_l = W_l h_l + b_l, h_{l+1} = relu(z_l) for
    l < L-1, output o = z_{L-1} (linear);
  * parameters are one flat vector: for each layer, W_l row-major
    (out_l x in_l), then b_l;
  * per-sample loss, averaged over the batch, for targets (y_0, y_1) and a
    mask (1 where y_0 is defined):
        mask * k(o_0 - y_0) * (o_0 - y_0)^2  +  lam * (softplus(o_1) - y_1 o_1),
    k(e) = kappa for e < 0 (under-prediction), 1 otherwise; the second term
    is the binary cross-entropy of sigmoid(o_1) against y_1;
  * the backward pass is the chain rule for the above;
  * Adam (Kingma and Ba, 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
    theta -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).

Pinned by tests/test_oracle_mlp.py: central finite differences of the loss
against the backward pass, a hand-built network with a known output, the
cross-entropy at o_1 = 0 (log 2 for any target), and the closed form of Adam
under a constant gradient.
"""
from __future__ import annotations

import numpy as np

SIZES = (12, 64, 64, 64, 2)   # input, three hidden layers of 64, output


def n_params(sizes=SIZES) -> int:
    return sum(sizes[i + 1] * sizes[i] + sizes[i + 1] for i in range(len(sizes) - 1))


def unpack(theta, sizes=SIZES):
    """Views (W_l, b_l) into the flat parameter vector."""
    out, off = [], 0
    for i in range(len(sizes) - 1):
        fi, fo = sizes[i], sizes[i + 1]
        W = theta[off: off + fo * fi].reshape(fo, fi)
        off += fo * fi
        b = theta[off: off + fo]
        off += fo
        out.append((W, b))
    assert off == theta.size
    return out


def init_params(seed: int, sizes=SIZES) -> np.ndarray:
    """He-normal weights, zero biases (float64)."""
    rng = np.random.default_rng(seed)
    parts = []
    for i in range(len(sizes) - 1):
        fi, fo = sizes[i], sizes[i + 1]
        parts.append(rng.standard_normal(fo * fi) * np.sqrt(2.0 / fi))
        parts.append(np.zeros(fo))
    return np.concatenate(parts)


def forward(theta, X, sizes=SIZES, dtype=np.float64, keep=False):
    """o = network(X) for a batch X (B x in).  With keep=True also returns the
    layer inputs h_l and pre-activations z_l for the backward pass."""
    th = np.asarray(theta, dtype=dtype)
    h = np.asarray(X, dtype=dtype)
    hs, zs = [], []
    layers = unpack(th, sizes)
    for l, (W, b) in enumerate(layers):
        hs.append(h)
        z = h @ W.T + b
        zs.append(z)
        h = np.maximum(z, 0) if l < len(layers) - 1 else z
    return (h, hs, zs) if keep else h


def softplus(z):
    """log(1 + e^z), evaluated without overflow."""
    return np.maximum(z, 0) + np.log1p(np.exp(-np.abs(z)))


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def loss(theta, X, Y, mask, lam=0.1, kappa=4.0, sizes=SIZES):
    o = forward(theta, X, sizes)
    e = o[:, 0] - Y[:, 0]
    k = np.where(e < 0, kappa, 1.0)
    per = mask * k * e * e + lam * (softplus(o[:, 1]) - Y[:, 1] * o[:, 1])
    return float(np.mean(per))


def loss_grad(theta, X, Y, mask, lam=0.1, kappa=4.0, sizes=SIZES):
    """(loss, gradient of the loss with respect to the flat parameters)."""
    o, hs, zs = forward(theta, X, sizes, keep=True)
    B = X.shape[0]
    e = o[:, 0] - Y[:, 0]
    k = np.where(e < 0, kappa, 1.0)
    per = mask * k * e * e + lam * (softplus(o[:, 1]) - Y[:, 1] * o[:, 1])
    # dL/do for every sample
    g = np.zeros_like(o)
    g[:, 0] = 2.0 * mask * k * e / B
    g[:, 1] = lam * (sigmoid(o[:, 1]) - Y[:, 1]) / B
    layers = unpack(np.asarray(theta, dtype=np.float64), sizes)
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        if l < len(layers) - 1:
            g = g * (zs[l] > 0)            # through relu(z_l)
        grads[l] = (g.T @ hs[l], g.sum(axis=0))
        g = g @ W                          # dL/dh_l
    flat = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    return float(np.mean(per)), flat


class Adam:
    """Adam with bias correction; state is float64."""

    def __init__(self, n, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, theta, g):
        self.t += 1
        self.m = self.b1 * self.m + (1.0 - self.b1) * g
        self.v = self.b2 * self.v + (1.0 - self.b2) * g * g
        mh = self.m / (1.0 - self.b1 ** self.t)
        vh = self.v / (1.0 - self.b2 ** self.t)
        return theta - self.lr * mh / (np.sqrt(vh) + self.eps)
