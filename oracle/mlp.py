"""Float64 reference of the learned block preconditioner's network.

A 3-layer perceptron  x -> relu(x W1^T + b1) -> relu(. W2^T + b2) -> . W3^T + b3
with bfloat16-valued weights (the GPU keeps float32 master weights and
computes with their bfloat16 rounding) and the mean-squared-error loss
  loss = 1/(2 B) sum_b |y_b - t_b|^2.
Forward and backward are written out plainly for gradient checks of the GPU
kernels; the functions are pinned by finite differences in
tests/test_oracle_mlp.py.  (The network is not part of the paper: it is the
learned component of this implementation, judged against plain Jacobi PCG.)
"""
import numpy as np


def bf16_round(a):
    """Round float values to the nearest bfloat16 (ties to even)."""
    f = np.asarray(a, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    bias = 0x7FFF + ((bits >> 16) & 1)
    out = ((bits + bias) & 0xFFFF0000).astype(np.uint32)
    return out.view(np.float32).astype(np.float64)


def init_params(n_in, width, n_out, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    p = {}
    dims = [(width, n_in), (width, width), (n_out, width)]
    for l, (o, i) in enumerate(dims, start=1):
        p[f"W{l}"] = rng.normal(0.0, np.sqrt(2.0 / i), size=(o, i))
        p[f"b{l}"] = np.zeros(o)
    return p


def forward_weights(W1, W2, W3, b1, b2, b3, x):
    """Forward pass with the given (already rounded) weights."""
    z1 = x @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3.T + b3
    return y, (x, z1, h1, z2, h2)


def forward(p, x):
    W1, W2, W3 = (bf16_round(p[k]) for k in ("W1", "W2", "W3"))
    return forward_weights(W1, W2, W3, p["b1"], p["b2"], p["b3"], x)


def loss(p, x, t):
    y, _ = forward(p, x)
    return 0.5 * float(np.sum((y - t) ** 2)) / x.shape[0]


def backward(p, x, t):
    """Gradients of loss w.r.t. the (float32 master) parameters; the weight
    rounding is treated as the identity (straight-through)."""
    y, (x, z1, h1, z2, h2) = forward(p, x)
    W2, W3 = bf16_round(p["W2"]), bf16_round(p["W3"])
    B = x.shape[0]
    dy = (y - t) / B
    g = {"W3": dy.T @ h2, "b3": dy.sum(0)}
    dh2 = (dy @ W3) * (z2 > 0)
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(0)
    dh1 = (dh2 @ W2) * (z1 > 0)
    g["W1"] = dh1.T @ x
    g["b1"] = dh1.sum(0)
    return g
