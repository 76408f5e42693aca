"""The cost model's network, written plainly in float64 numpy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper has no learned model (it fixes its parameters by the noise analysis
of Sec. 3.2.1); this is the reference for the GPU network that ranks layer
configurations by predicted time.  Definitions:

  * network: F features -> 64 -> 64 -> 1, ReLU after each hidden layer;
    inputs standardised as (x - mean) / std, output destandardised as
    y * std_y + mean_y;
  * loss: mean over a mini-batch of (net(x) - (y - mean_y) / std_y)^2;
  * Adam (Kingma and Ba, ICLR 2015): m = b1 m + (1 - b1) g,
    v = b2 v + (1 - b2) g^2, p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps);
  * mini-batch slot j of step t draws row SplitMix64(seed xor SplitMix64(t 2^32 + t + j)) mod n,
    where SplitMix64(z) is the published generator's output for state z
    (Steele, Lea and Flood, OOPSLA 2014).

Parameter vector (as the library stores it): W1[64][F], b1[64], W2[64][64],
b2[64], w3[64], b3, mean[F], mean_y, std[F], std_y.
"""
from __future__ import annotations

import numpy as np

H = 64
MASK = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def splitmix64(z: int) -> int:
    """Output of SplitMix64 whose state before the step is z."""
    z = (z + GAMMA) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def n_weights(F: int) -> int:
    return H * F + H + H * H + H + H + 1


def unpack(params: np.ndarray, F: int) -> dict:
    p = np.asarray(params, dtype=np.float64)
    o = 0
    out = {}
    for name, shape in (("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", ())):
        size = int(np.prod(shape)) if shape else 1
        out[name] = p[o:o + size].reshape(shape) if shape else p[o]
        o += size
    out["xm"], out["ym"] = p[o:o + F], p[o + F]
    o += F + 1
    out["xs"], out["ys"] = p[o:o + F], p[o + F]
    return out


def hidden(P: dict, X: np.ndarray):
    """Standardised inputs and the two hidden layers' activations, row per sample."""
    Z = (np.asarray(X, dtype=np.float64) - P["xm"]) / P["xs"]
    A1 = Z @ P["W1"].T + P["b1"]
    H1 = np.maximum(A1, 0.0)
    A2 = H1 @ P["W2"].T + P["b2"]
    H2 = np.maximum(A2, 0.0)
    return Z, H1, H2


def predict(params: np.ndarray, F: int, X: np.ndarray) -> np.ndarray:
    P = unpack(params, F)
    _, _, H2 = hidden(P, X)
    return (H2 @ P["w3"] + P["b3"]) * P["ys"] + P["ym"]


def batch_rows(seed: int, step: int, batch: int, n: int) -> np.ndarray:
    return np.array([splitmix64(seed ^ splitmix64((step * 0x100000001 + j) & MASK)) % n for j in range(batch)])


def loss_and_grad(params: np.ndarray, F: int, X: np.ndarray, y: np.ndarray, rows: np.ndarray):
    """Mean squared error of the standardised target over `rows` and its gradient with
    respect to the weights (the first n_weights(F) entries), by back-propagation."""
    P = unpack(params, F)
    Xb, yb = np.asarray(X, dtype=np.float64)[rows], np.asarray(y, dtype=np.float64)[rows]
    Z, H1, H2 = hidden(P, Xb)
    out = H2 @ P["w3"] + P["b3"]
    err = out - (yb - P["ym"]) / P["ys"]
    B = len(rows)
    loss = float(np.mean(err ** 2))
    dy = 2.0 * err / B                              # d loss / d out, per sample
    g_w3 = H2.T @ dy
    g_b3 = dy.sum()
    d2 = np.outer(dy, P["w3"]) * (H2 > 0)           # d loss / d A2
    g_W2 = d2.T @ H1
    g_b2 = d2.sum(axis=0)
    d1 = (d2 @ P["W2"]) * (H1 > 0)                  # d loss / d A1
    g_W1 = d1.T @ Z
    g_b1 = d1.sum(axis=0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return loss, g


def adam(w: np.ndarray, m: np.ndarray, v: np.ndarray, g: np.ndarray, t: int, lr: float,
         b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam step (t counts from 1); returns the new (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh, vh = m / (1 - b1 ** t), v / (1 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def scaling(X: np.ndarray, y: np.ndarray):
    """Column means and population standard deviations (floor 1e-6) of X and of y."""
    X, y = np.asarray(X, dtype=np.float64), np.asarray(y, dtype=np.float64)
    return (X.mean(axis=0), y.mean(), np.maximum(X.std(axis=0), 1e-6), max(float(y.std()), 1e-6))
