"""Pins of the cost model's reference network (oracle/mlp.py) against facts
that do not come from it: the published SplitMix64 outputs, central finite
differences of the loss, closed forms of the forward pass and of Adam's
first step."""
import numpy as np

from oracle import mlp


def _params(F, rng, scale=0.5):
    w = rng.normal(0.0, scale, mlp.n_weights(F))
    xm, xs = rng.normal(0, 1, F), rng.uniform(0.5, 2.0, F)
    return np.concatenate([w, xm, [0.7], xs, [1.3]])


def test_splitmix64_published_outputs():
    # the generator's first three outputs from state 0 (Steele, Lea and Flood's SplitMix64)
    g = mlp.GAMMA
    assert mlp.splitmix64(0) == 0xE220A8397B1DCDAF
    assert mlp.splitmix64(g) == 0x6E789E6AA1B965F4
    assert mlp.splitmix64((2 * g) & mlp.MASK) == 0x06C45D188009454F


def test_batch_rows_in_range_and_reproducible():
    a = mlp.batch_rows(5, 3, 100, 37)
    assert a.min() >= 0 and a.max() < 37
    assert (a == mlp.batch_rows(5, 3, 100, 37)).all()
    assert not (a == mlp.batch_rows(5, 4, 100, 37)).all()


def test_gradient_matches_central_differences():
    F, n = 5, 40
    rng = np.random.default_rng(0)
    p = _params(F, rng)
    X, y = rng.normal(0, 1, (n, F)), rng.normal(0, 1, n)
    rows = mlp.batch_rows(11, 0, 9, n)
    loss, g = mlp.loss_and_grad(p, F, X, y, rows)
    assert g.shape == (mlp.n_weights(F),)
    eps = 1e-6
    for i in rng.choice(mlp.n_weights(F), 120, replace=False).tolist() + [mlp.n_weights(F) - 1]:
        q = p.copy()
        q[i] += eps
        lp, _ = mlp.loss_and_grad(q, F, X, y, rows)
        q[i] -= 2 * eps
        lm, _ = mlp.loss_and_grad(q, F, X, y, rows)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_forward_closed_forms():
    F = 3
    X = np.array([[1.5, -2.0, 0.3], [-0.5, 4.0, 1.0]])
    p = np.zeros(mlp.n_weights(F) + 2 * (F + 1))
    o = mlp.n_weights(F)
    p[o + F + 1:o + 2 * F + 2] = 1.0                 # unit standard deviations
    p[mlp.n_weights(F) - 1] = 0.25                   # b3
    p[o + F], p[o + 2 * F + 1] = 2.0, 3.0            # mean_y, std_y
    assert np.allclose(mlp.predict(p, F, X), 3.0 * 0.25 + 2.0)
    # a single active path: out = relu(relu(x0)) * 1 (W1[0][0] = W2[0][0] = w3[0] = 1)
    q = np.zeros_like(p)
    q[o + F + 1:o + 2 * F + 2] = 1.0
    q[0] = 1.0                                       # W1[0][0]
    q[mlp.H * F + mlp.H] = 1.0                       # W2[0][0]
    q[mlp.H * F + mlp.H + mlp.H * mlp.H + mlp.H] = 1.0  # w3[0]
    assert np.allclose(mlp.predict(q, F, X), [1.5, 0.0])


def test_adam_first_step_is_lr_times_sign():
    rng = np.random.default_rng(1)
    w, g = rng.normal(0, 1, 50), rng.normal(0, 1, 50)
    w1, m1, v1 = mlp.adam(w, np.zeros(50), np.zeros(50), g, 1, 0.01)
    assert np.allclose(w1, w - 0.01 * g / (np.abs(g) + 1e-8))
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)


def test_loss_of_constant_network():
    F, n = 2, 10
    rng = np.random.default_rng(2)
    X, y = rng.normal(0, 1, (n, F)), rng.normal(5, 2, n)
    p = np.zeros(mlp.n_weights(F) + 2 * (F + 1))
    o = mlp.n_weights(F)
    p[o + F + 1:] = 1.0
    p[o + F], p[o + 2 * F + 1] = 5.0, 2.0
    rows = np.arange(n)
    loss, _ = mlp.loss_and_grad(p, F, X, y, rows)
    assert np.isclose(loss, np.mean(((y - 5.0) / 2.0) ** 2))


def test_scaling_is_population_moments():
    X = np.array([[1.0, 5.0], [3.0, 5.0]])
    xm, ym, xs, ys = mlp.scaling(X, np.array([2.0, 4.0]))
    assert np.allclose(xm, [2.0, 5.0]) and ym == 3.0
    assert np.allclose(xs, [1.0, 1e-6]) and ys == 1.0
