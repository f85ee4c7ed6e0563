"""Pins of the numpy reference of the surrogate network: the convolution against
its definition on small cases, the (un)shuffle as an exact inverse pair, and
every parameter gradient against central finite differences."""
import numpy as np
import pytest

from oracle import surrogate as S


def test_conv_matches_definition():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 7, 3))
    W = rng.normal(size=(4, 5, 3))
    b = rng.normal(size=4)
    y = S.conv(x, W, b)
    for n in range(2):
        for l in range(7):
            for o in range(4):
                acc = b[o]
                for t in range(5):
                    q = l + t - 2
                    if 0 <= q < 7:
                        acc += W[o, t] @ x[n, q]
                assert abs(y[n, l, o] - acc) < 1e-12


def test_shuffle_inverts_unshuffle():
    x = np.arange(2 * 16 * 3, dtype=float).reshape(2, 16, 3)
    q = S.unshuffle(x)
    assert q.shape == (2, 4, 12)
    assert q[0, 1, 3 * 2 + 1] == x[0, 4 * 1 + 2, 1]  # fine p = R q + r -> channel r Cin + c
    np.testing.assert_array_equal(S.shuffle(q, 3), x)


def test_conv_backward_is_adjoint():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 9, 3))
    W = rng.normal(size=(4, 5, 3))
    dy = rng.normal(size=(2, 9, 4))
    dx, dW, db = S.conv_backward(x, W, dy)
    y = S.conv(x, W, np.zeros(4))
    # <dy, conv(x)> = <dx, x> for the linear map x -> conv(x)
    assert abs((dy * y).sum() - (dx * x).sum()) < 1e-10
    assert abs((dy * y).sum() - (dW * W).sum()) < 1e-10
    np.testing.assert_allclose(db, dy.sum((0, 1)))


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    cin, cout, width, nb = 3, 2, 6, 2
    p = S.init_params(cin, cout, width, nb, seed=3)
    for k in p:
        if k.endswith("_b") or "_b" in k.split("_")[-1]:
            p[k] = rng.normal(0, 0.1, p[k].shape)
    x = rng.normal(size=(2, 16, cin))
    target = rng.normal(size=(2, 16, cout))
    mask = (rng.uniform(size=(2, 16)) > 0.3).astype(float)
    loss, g, _ = S.loss_and_grad(p, x, target, mask, nb, cout)
    eps = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _, _ = S.loss_and_grad(p, x, target, mask, nb, cout)
            flat[idx] = old - eps
            lm, _, _ = S.loss_and_grad(p, x, target, mask, nb, cout)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            an = g[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (k, idx, fd, an)


def test_bf16_rounding_matches_library_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.normal(size=4000) * 10.0 ** rng.integers(-6, 6, size=4000),
                        [0.0, -0.0, 1.0, -3.5, 65504.0, 1e-30]])
    # exact ties between two bfloat16 neighbours: mantissa ...1 1000 0000 0000 0000 and ...0 1000 ...
    ties = (np.array([0x3F818000, 0x3F808000, 0xBF818000, 0x40A08000], dtype=np.uint32)
            .view(np.float32).astype(np.float64))
    x = np.concatenate([x, ties])
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(S.bf16(x), ref.astype(np.float64))
    # rounding a bfloat16 value is the identity
    np.testing.assert_array_equal(S.bf16(S.bf16(x)), S.bf16(x))


def test_flatten_roundtrip_and_layout():
    p = S.init_params(3, 2, 16, 2, seed=5)
    v = S.flatten(p, 2)
    assert v.size == sum(a.size for a in p.values())
    q = S.unflatten(v, 3, 2, 16, 2)
    for k in p:
        np.testing.assert_array_equal(p[k], q[k])
    # the first layer's weights lead, in W[o][t][i] order, followed by its biases
    np.testing.assert_array_equal(v[:p["lift_w"].size], p["lift_w"].reshape(-1))
    n = p["lift_w"].size
    np.testing.assert_array_equal(v[n:n + 16], p["lift_b"])


def test_adam_first_step_moves_by_lr_times_sign():
    # with bias correction the first step is lr * g / (|g| + eps) per entry
    rng = np.random.default_rng(6)
    g = {"a": rng.normal(size=50) * 10.0 ** rng.integers(-3, 3, size=50)}
    p = {"a": np.zeros(50)}
    m = {"a": np.zeros(50)}
    v = {"a": np.zeros(50)}
    S.adam(p, g, m, v, 1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(p["a"], -0.01 * np.sign(g["a"]), rtol=1e-12)
    # constant gradient: every step is again lr * sign(g) (m-hat = g, v-hat = g^2)
    for step in range(2, 6):
        S.adam(p, g, m, v, step, lr=0.01, eps=0.0)
    np.testing.assert_allclose(p["a"], -0.05 * np.sign(g["a"]), rtol=1e-10)
