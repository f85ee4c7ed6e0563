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


def _tube_block(nx, rng):
    rho = rng.uniform(0.2, 1.0, 2 * nx)
    return np.stack([rho, rng.normal(0, 0.2, 2 * nx), rng.uniform(0.15, 0.4, 2 * nx),
                     rho * rng.uniform(0.15, 0.4, 2 * nx)])


def test_conserved_primitive_inverse_and_energy():
    rng = np.random.default_rng(7)
    v = _tube_block(9, rng)
    np.testing.assert_allclose(S.primitive(S.conserved(v)), v, rtol=1e-13)
    # one point by hand: rho 2, u 0.5, theta 0.3, E_R 0.4 -> E = 0.25 + 0.9 + 0.4
    U = S.conserved(np.array([2.0, 0.5, 0.3, 0.4]))
    np.testing.assert_allclose(U, [2.0, 1.0, 1.55, 0.4], rtol=1e-15)


def test_position_order_interleaves_sublattices():
    blk = np.arange(4 * 6, dtype=float).reshape(4, 6)  # nx = 3: points (s=0, x=0..2), (s=1, x=0..2)
    seq = S.position_order(blk, 3)
    np.testing.assert_array_equal(seq[0], [0, 3, 1, 4, 2, 5])
    np.testing.assert_array_equal(S.point_order(seq, 3), blk)


def test_pack_padding_and_features():
    rng = np.random.default_rng(8)
    nx, pad = 5, 4
    src = _tube_block(nx, rng)
    res = np.array([[1.0, 0.0, 0.3, 0.3], [0.5, 0.0, 0.25, 0.12]])
    x, _, _ = S.pack(src, None, nx, res, (0.7, -0.2), pad, 0, 2 * nx + 2 * pad, 0,
                     (0, 0, 0, 0), (1, 1, 1, 1), (1, 1, 1, 1))
    assert np.all(x[:pad, 10] == 0) and np.all(x[pad:pad + 2 * nx, 10] == 1) and np.all(x[pad + 2 * nx:, 10] == 0)
    assert np.all(x[:, 4:8] == 0)  # no previous window
    np.testing.assert_allclose(x[:pad, :4], np.broadcast_to(res[0], (pad, 4)), rtol=1e-7)
    np.testing.assert_allclose(x[pad + 2 * nx:, :4], np.broadcast_to(res[1], (pad, 4)), rtol=1e-7)
    np.testing.assert_allclose(x[pad:pad + 2 * nx, :4].T, S.position_order(src, nx), rtol=1e-7)
    np.testing.assert_allclose(x[:, 8:10], np.broadcast_to([0.7, -0.2], (2 * nx + 2 * pad, 2)), rtol=1e-7)
    prev = src * 0.9
    x2, _, _ = S.pack(src, None, nx, res, (0.7, -0.2), pad, 0, 2 * nx + 2 * pad, 0,
                      (0, 0, 0, 0), (1, 1, 1, 1), (1, 1, 1, 1), prev=prev, dscale=(2, 2, 2, 2))
    np.testing.assert_allclose(x2[pad:pad + 2 * nx, 4:8].T, S.position_order(0.05 * src, nx), rtol=1e-5)
    assert np.all(x2[:pad, 4:8] == 0) and np.all(x2[pad + 2 * nx:, 4:8] == 0)


def test_apply_inverts_pack_targets():
    # the increments pack builds from (src, tgt), applied to src without
    # projection, give back tgt
    rng = np.random.default_rng(9)
    nx, pad, crop = 7, 4, 2
    src, tgt = _tube_block(nx, rng), _tube_block(nx, rng)
    out_scale = (0.1, 0.05, 0.2, 0.03)
    length = 2 * nx + 2 * pad - crop
    _, t, mask = S.pack(src, tgt, nx, np.ones((2, 4)), (0, 0), pad, crop, length, 0,
                        (0, 0, 0, 0), (1, 1, 1, 1), out_scale)
    assert mask.sum() == 2 * nx
    new, bad, tot = S.apply(src, t, nx, pad, crop, out_scale, project=False)
    assert not bad
    np.testing.assert_allclose(new, tgt, rtol=1e-12, atol=1e-14)
    assert abs(tot[0] - tgt[0].sum()) < 1e-12


def test_apply_projection_conserves_mass_and_energy():
    rng = np.random.default_rng(10)
    nx, pad = 11, 0
    src = _tube_block(nx, rng)
    y = rng.normal(0, 1, (2 * nx, 4))
    out_scale = (0.01, 0.01, 0.01, 0.005)
    new, bad, tot = S.apply(src, y, nx, pad, 0, out_scale, project=True)
    U0, U1 = S.conserved(src), S.conserved(new)
    assert abs(U1[0].sum() - U0[0].sum()) < 1e-12 and abs(U1[2].sum() - U0[2].sum()) < 1e-12
    assert abs(tot[0] - U0[0].sum()) < 1e-12 and abs(tot[1] - U0[2].sum()) < 1e-12
    # momentum and E_R increments are left alone
    d = S.position_order(U1 - U0, nx)
    np.testing.assert_allclose(d[1], 0.01 * y[:, 1], atol=1e-12)
    np.testing.assert_allclose(d[3], 0.005 * y[:, 3], atol=1e-12)
    # increments that already sum to zero are unchanged
    y2 = y.copy()
    y2[:, 0] -= y2[:, 0].mean()
    y2[:, 2] -= y2[:, 2].mean()
    a, _, _ = S.apply(src, y2, nx, pad, 0, out_scale, project=True)
    b, _, _ = S.apply(src, y2, nx, pad, 0, out_scale, project=False)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-14)
    # a negative density is reported
    y3 = np.zeros((2 * nx, 4))
    y3[3, 0] = -1e3
    assert S.apply(src, y3, nx, pad, 0, out_scale, project=False)[1]


def test_splitmix64_reference_values():
    # first outputs of SplitMix64 seeded with 0, as published with the generator
    assert S.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert S.splitmix64(0, 1) == 0x6E789E6AA1B965F4
    assert S.splitmix64(0, 2) == 0x06C45D188009454F


def test_pack_noise_perturbs_source_state():
    rng = np.random.default_rng(11)
    nx, pad = 6, 4
    src, tgt = _tube_block(nx, rng), _tube_block(nx, rng)
    args = (src, tgt, nx, np.ones((2, 4)), (0, 0), pad, 0, 2 * nx + 2 * pad, 0, (0, 0, 0, 0), (1, 1, 1, 1),
            (1, 1, 1, 1))
    x0, t0, _ = S.pack(*args)
    x1, t1, _ = S.pack(*args, noise=(1e-2, 0, 0, 2e-3), seed=7)
    d = x1[:, :4] - x0[:, :4]
    assert np.all(d[:pad] == 0) and np.all(d[pad + 2 * nx:] == 0)  # padding is not perturbed
    assert np.all(d[:, 1:3] == 0)
    assert 0 < np.abs(d[pad:pad + 2 * nx, 0]).max() <= 1.8e-2
    # the target undoes the perturbation: U(tgt) - U(v + e) for rho is the old target minus e
    np.testing.assert_allclose(t1[pad:pad + 2 * nx, 0], t0[pad:pad + 2 * nx, 0] - d[pad:pad + 2 * nx, 0],
                               atol=1e-6)
