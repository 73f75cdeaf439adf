"""Oracle network of the learned preconditioner: gradients equal finite
differences of the loss (with the bf16 weight rounding held fixed), and
bf16 rounding matches the definition (8 significant bits, ties to even)."""
import numpy as np

from oracle.mlp import backward, bf16_round, forward, forward_weights, init_params, loss


def test_bf16_rounding():
    assert bf16_round(1.0) == 1.0
    assert bf16_round(1.0 + 2 ** -9) == 1.0            # tie -> even
    assert bf16_round(1.0 + 3 * 2 ** -9) == 1.0 + 2 ** -7
    x = np.random.default_rng(0).normal(size=1000)
    r = bf16_round(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2 ** -8 + 1e-300)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    p = init_params(6, 16, 3, seed=2)
    # move master weights onto the bf16 grid so that rounding is inert under +-h
    for k in ("W1", "W2", "W3"):
        p[k] = bf16_round(p[k])
    x = rng.normal(size=(9, 6))
    t = rng.normal(size=(9, 3))
    g = backward(p, x, t)
    h = 1e-6
    for k in ("b1", "b2", "b3"):
        for idx in np.ndindex(p[k].shape):
            q = {kk: v.copy() for kk, v in p.items()}
            q[k][idx] += h
            lp = loss(q, x, t)
            q[k][idx] -= 2 * h
            lm = loss(q, x, t)
            assert abs((lp - lm) / (2 * h) - g[k][idx]) < 1e-6
    # weight gradients: finite differences on the weights the forward pass uses
    Ws = {k: bf16_round(p[k]) for k in ("W1", "W2", "W3")}

    def L(W):
        y, _ = forward_weights(W["W1"], W["W2"], W["W3"], p["b1"], p["b2"], p["b3"], x)
        return 0.5 * float(np.sum((y - t) ** 2)) / x.shape[0]

    for k in ("W1", "W2", "W3"):
        for idx in list(np.ndindex(p[k].shape))[::7]:
            q = {kk: v.copy() for kk, v in Ws.items()}
            q[k][idx] += h
            lp = L(q)
            q[k][idx] -= 2 * h
            lm = L(q)
            assert abs((lp - lm) / (2 * h) - g[k][idx]) < 1e-6, (k, idx)


def test_forward_hand_computed():
    """x -> relu(x W1^T + b1) -> relu(. W2^T + b2) -> . W3^T + b3 on values
    exact in bf16, worked by hand: z1 = (1, -2, -0.5) -> h1 = (1, 0, 0);
    z2 = (1, 1, 0) -> h2 = (1, 1, 0); y = 1 + 2 - 1 = 2.  The weights the
    forward pass uses are the bf16 roundings of the masters."""
    p = {"W1": np.array([[1.0, 0.0], [0.0, 1.0], [1.0, 1.0]]), "b1": np.array([0.0, 0.0, 0.5]),
         "W2": np.eye(3), "b2": np.array([0.0, 1.0, 0.0]),
         "W3": np.array([[1.0, 2.0, 3.0]]), "b3": np.array([-1.0])}
    x = np.array([[1.0, -2.0]])
    y, (_, z1, h1, z2, h2) = forward(p, x)
    assert np.array_equal(z1, [[1.0, -2.0, -0.5]]) and np.array_equal(h1, [[1.0, 0.0, 0.0]])
    assert np.array_equal(z2, [[1.0, 1.0, 0.0]]) and np.array_equal(h2, [[1.0, 1.0, 0.0]])
    assert np.array_equal(y, [[2.0]])
    q = dict(p)
    q["W3"] = p["W3"] + np.array([[2 ** -9, 0.0, 0.0]])     # rounds back to 1.0 (tie to even)
    assert np.array_equal(forward(q, x)[0], [[2.0]])
    assert loss(p, x, np.array([[0.5]])) == 0.5 * 1.5 ** 2
