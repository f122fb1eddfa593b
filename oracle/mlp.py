"""ORACLE -- test infrastructure only.

Plain numpy (float64) reference of the learned work model's network: a
4 -> 32 -> 32 -> 1 perceptron with ReLU hidden layers, parameters packed as
W1[32][4], b1[32], W2[32][32], b2[32], W3[32], b3 (1249 values), mean squared
error loss.  Forward and hand-derived backward passes, used to check the
CUDA kernels' outputs and gradients."""
import numpy as np

NIN, NH = 4, 32
SIZES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH,)),
         ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, off = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = p[off:off + k].reshape(shape)
        off += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SIZES])


def forward(p, X):
    w = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ w["W1"].T + w["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w["W3"] + w["b3"][0]
    return y, (X, z1, h1, z2, h2)


def loss_and_grad(p, X, T):
    """Mean squared error and its gradient with respect to the packed params."""
    w = unpack(p)
    y, (X, z1, h1, z2, h2) = forward(p, X)
    T = np.asarray(T, dtype=np.float64)
    N = X.shape[0]
    e = y - T
    loss = float((e * e).mean())
    dy = 2.0 * e / N
    g = {"W3": h2.T @ dy, "b3": np.array([dy.sum()])}
    d2 = np.outer(dy, w["W3"]) * (z2 > 0)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(0)
    d1 = (d2 @ w["W2"]) * (z1 > 0)
    g["W1"] = d1.T @ X
    g["b1"] = d1.sum(0)
    return loss, pack(g)


def init(seed):
    """He-uniform initialisation (float32 values)."""
    rng = np.random.default_rng(seed)
    d = {"W1": rng.uniform(-1, 1, (NH, NIN)) * np.sqrt(6.0 / NIN),
         "b1": np.zeros(NH), "W2": rng.uniform(-1, 1, (NH, NH)) * np.sqrt(6.0 / NH),
         "b2": np.zeros(NH), "W3": rng.uniform(-1, 1, NH) * np.sqrt(3.0 / NH),
         "b3": np.zeros(1)}
    return pack(d).astype(np.float32)
