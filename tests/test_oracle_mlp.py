"""Pins of the proposal-network oracle: the backward pass equals central finite
differences of the listwise loss; the loss is the cross-entropy a uniform
scorer gives (log n) when all weights vanish; bfloat16 rounding is exact on
representable values and rounds half to even."""
import numpy as np

from oracle import mlp


def _data(rng, events=40):
    sizes = rng.integers(1, 7, size=events)
    offsets = np.concatenate([[0], np.cumsum(sizes)])
    X = rng.normal(size=(offsets[-1], mlp.NF))
    labels = np.array([rng.integers(0, s) for s in sizes])
    return X, offsets, labels


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    X, off, lab = _data(rng)
    theta = mlp.init(seed=1)
    loss, g = mlp.loss_and_grad(theta, X, off, lab)
    h = 1e-6
    idx = rng.choice(mlp.NPARAM, 200, replace=False)
    # include every block of parameters
    idx = np.concatenate([idx, [0, mlp.NF * mlp.H - 1, 16 * 64 + 3, 16 * 64 + 64 + 100,
                                mlp.NPARAM - 66, mlp.NPARAM - 2, mlp.NPARAM - 1]])
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (mlp.loss_and_grad(tp, X, off, lab)[0] - mlp.loss_and_grad(tm, X, off, lab)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])
    # padded input rows carry no gradient
    p = mlp.unpack(g)
    assert np.all(p["W1"][mlp.NF:] == 0)


def test_zero_network_gives_uniform_choice():
    rng = np.random.default_rng(4)
    X, off, lab = _data(rng)
    theta = np.zeros(mlp.NPARAM)
    loss, _ = mlp.loss_and_grad(theta, X, off, lab)
    sizes = np.diff(off)
    assert abs(loss - np.mean(np.log(sizes))) < 1e-12


def test_training_reduces_loss_on_learnable_rule():
    # label = candidate with the smallest first feature: learnable by the MLP
    rng = np.random.default_rng(5)
    X, off, _ = _data(rng, events=200)
    lab = np.array([np.argmin(X[off[e]:off[e + 1], 0]) for e in range(len(off) - 1)])
    theta = mlp.init(seed=2)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    l0 = mlp.loss_and_grad(theta, X, off, lab)[0]
    for t in range(1, 301):
        loss, g = mlp.loss_and_grad(theta, X, off, lab)
        theta, m, v = mlp.adam_step(theta, g, m, v, t, lr=3e-3)
    assert loss < 0.5 * l0


def test_bf16_rounding():
    vals = np.array([1.0, -2.5, 0.0, 2.0 ** 127, -0.15625], dtype=np.float32)
    assert np.array_equal(mlp.bf16_round(vals), vals)
    # 1 + 2^-8 lies halfway between bf16 neighbours 1 and 1 + 2^-7: ties to even (1)
    assert mlp.bf16_round(np.float32(1 + 2 ** -8)) == 1.0
    assert mlp.bf16_round(np.float32(1 + 3 * 2 ** -8)) == np.float32(1 + 2 ** -6)


def _representable_case(rng):
    """Operands on which every BF16 rounding is exact: inputs in {0, +-1/2, +-1},
    W1 in quarters, sparse W2 in {0, +-1/2}, w3 in {+-1/2, +-1}; two events of
    two candidates that differ only in feature 11, whose W1 row is zero, so
    both candidates tie (softmax 1/2) and the back-propagated values stay on
    a coarse dyadic grid."""
    p = {"W1": np.zeros((mlp.KPAD, mlp.H)), "b1": np.zeros(mlp.H), "W2": np.zeros((mlp.H, mlp.H)),
         "b2": np.zeros(mlp.H), "w3": rng.choice([-1.0, -0.5, 0.5, 1.0], mlp.H), "b3": np.array([0.25])}
    p["W1"][:11] = rng.integers(-4, 5, (11, mlp.H)) / 4.0
    p["b1"][:] = rng.integers(-4, 5, mlp.H) / 8.0
    for m in range(mlp.H):
        cols = rng.choice(mlp.H, 4, replace=False)
        p["W2"][m, cols] = rng.choice([-0.5, 0.5], 4)
    X = np.zeros((4, mlp.NF))
    for e in range(2):
        base = rng.choice([-1.0, -0.5, 0.0, 0.5, 1.0], mlp.NF)
        X[2 * e] = base
        X[2 * e + 1] = base
        X[2 * e, 11], X[2 * e + 1, 11] = 1.0, -1.0
    return mlp.pack(p), X, np.array([0, 2, 4]), np.array([0, 1])


def test_bf16_operand_variant_is_exact_on_representable_operands():
    rng = np.random.default_rng(12)
    theta, X, off, lab = _representable_case(rng)
    loss, g = mlp.loss_and_grad(theta, X, off, lab)
    loss_b, y_b, g_b = mlp.loss_and_grad_bf16(theta, X, off, lab)
    y, _ = mlp.forward(theta, X)
    assert np.array_equal(y, y_b) and loss == loss_b
    assert np.array_equal(g, g_b)
    assert abs(loss - np.log(2.0)) < 1e-15          # both candidates tie
    assert np.abs(g).max() > 0.0 and np.abs(g[11 * mlp.H:12 * mlp.H]).max() > 0.0


def test_bf16_operand_variant_error_is_of_bf16_size():
    rng = np.random.default_rng(13)
    X, off, lab = _data(rng, events=60)
    theta = mlp.init(seed=2)
    y, _ = mlp.forward(theta, X)
    _, y_b, _ = mlp.loss_and_grad_bf16(theta, X, off, lab)
    rel = np.abs(y_b - y).max() / np.abs(y).max()
    assert 1e-5 < rel < 3e-2
