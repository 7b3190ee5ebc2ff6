"""FP64 CPU oracle of the learned warm start's network: a multilayer
perceptron 3 -> 256 -> 256 -> 256 -> 64 with tanh hidden units and a linear
output, trained by mean squared error with Adam.

TEST INFRASTRUCTURE ONLY: imported by tests/ (gradient parity of the CUDA
forward and backward kernels, finite-difference pins).  Plain numpy, no
blocking or fusion; it shares no code with the CUDA library.

The paper does not use a network; the warm start is this project's
addition.  What the network predicts follows the paper's description of
the equilibrium shape (App. B): the radial profile r = G(phi) of the
droplet surface about its centre, phi the polar angle from the z axis,
made dimensionless as g = G / R0, sampled at 64 polar angles
phi_k = (k + 1/2) pi / 64.

Inputs: (theta_eq in degrees, R0, lambda), mapped to the features
u = ((theta_eq - 90) / 70, (R0 - 16) / 8, log10(lambda)).

Parameters are one flat vector, layer by layer: W_l (out_l x in_l, row
major) then b_l (out_l), for l = 0..3.
"""
from __future__ import annotations

import numpy as np

SIZES = (3, 256, 256, 256, 64)
NPHI = 64
BETA1, BETA2, EPS = 0.9, 0.999, 1e-8


def n_params(sizes=SIZES):
    return sum(o * i + o for i, o in zip(sizes[:-1], sizes[1:]))


def unpack(p, sizes=SIZES):
    """Views (W_l, b_l) into the flat parameter vector."""
    out, k = [], 0
    for i, o in zip(sizes[:-1], sizes[1:]):
        W = p[k:k + o * i].reshape(o, i)
        k += o * i
        b = p[k:k + o]
        k += o
        out.append((W, b))
    assert k == p.size
    return out


def features(x):
    """x: S x 3 raw inputs (theta_eq deg, R0, lambda) -> S x 3 features."""
    x = np.asarray(x, np.float64)
    return np.stack([(x[:, 0] - 90.0) / 70.0, (x[:, 1] - 16.0) / 8.0, np.log10(x[:, 2])], axis=1)


def forward(p, x, sizes=SIZES):
    """Returns (prediction S x 64, activations [u, h1, h2, h3])."""
    layers = unpack(np.asarray(p, np.float64), sizes)
    a = features(x)
    acts = [a]
    for l, (W, b) in enumerate(layers):
        z = a @ W.T + b
        a = np.tanh(z) if l < len(layers) - 1 else z
        if l < len(layers) - 1:
            acts.append(a)
    return a, acts


def loss(p, x, y, sizes=SIZES):
    """Mean squared error over all S x 64 outputs."""
    yhat, _ = forward(p, x, sizes)
    d = yhat - np.asarray(y, np.float64)
    return float(np.mean(d * d))


def grad(p, x, y, sizes=SIZES):
    """Gradient of loss() with respect to the flat parameters (backward
    pass by the chain rule, layer by layer)."""
    p = np.asarray(p, np.float64)
    layers = unpack(p, sizes)
    yhat, acts = forward(p, x, sizes)
    S, n_out = yhat.shape
    g = np.zeros_like(p)
    gl = unpack(g, sizes)
    dz = 2.0 * (yhat - np.asarray(y, np.float64)) / (S * n_out)   # d loss / d output
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        a_in = acts[l]
        gl[l][0][:] = dz.T @ a_in
        gl[l][1][:] = dz.sum(axis=0)
        if l > 0:
            dh = dz @ W
            dz = dh * (1.0 - acts[l] * acts[l])    # tanh' = 1 - tanh^2
    return g


class Adam:
    """Adam with bias correction: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
    p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)."""

    def __init__(self, n, lr):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr = lr

    def step(self, p, g):
        self.t += 1
        self.m = BETA1 * self.m + (1.0 - BETA1) * g
        self.v = BETA2 * self.v + (1.0 - BETA2) * g * g
        mh = self.m / (1.0 - BETA1 ** self.t)
        vh = self.v / (1.0 - BETA2 ** self.t)
        return p - self.lr * mh / (np.sqrt(vh) + EPS)
