"""FP64 numpy reference of the learned surrogate network (TEST INFRASTRUCTURE:
only tests may import it; the CUDA library never does).

The surrogate maps the moment fields of a quasi-1-D tube at step t to step
t + 32. The paper has no learned component; this network is the 1-D
convolutional operator of the build: on a sequence of L fine points with Cin
channels (L a multiple of R),
  unshuffle   (L, Cin)      -> (L/R, R*Cin)       position p = R*q + r -> channel r*Cin + c
  lift        conv k=1      (R*Cin -> C), bias
  blocks      x + conv5(relu(conv5(relu(x))))   (C -> C, kernel 5, zero padding), B times
  head        conv k=1      (C -> R*Cout), bias, after relu
  shuffle     (L/R, R*Cout) -> (L, Cout)
so the output is an increment added to the input state by the caller. Every
conv is y[q][o] = b[o] + sum_{t, i} W[o][t][i] x[q + t - (k-1)/2][i] with x = 0
outside the sequence. Written as plain loops over taps with einsum for the
channel contraction, forward and backward (reverse-mode by hand).

``rnd`` (optional) is applied to both operands of every contraction: passing
``bf16`` gives the operand rounding of a tensor-core evaluation with BF16
inputs (the products and sums stay FP64), so that such an evaluation can be
compared at a tolerance set by its FP32 accumulation alone.
"""
import numpy as np

R, K5 = 4, 5


def _ident(a):
    return a


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), via the float32 value:
    keep the upper 16 bits of the float32 pattern after adding 0x7fff plus the
    lowest kept bit. Non-finite inputs are not expected."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(a))


def init_params(cin, cout, width, nblocks, seed=0):
    """He-style initial weights (the CUDA library draws its own; tests copy
    parameters explicitly between the two)."""
    rng = np.random.default_rng(seed)
    p = {"lift_w": rng.normal(0, np.sqrt(2.0 / (R * cin)), (width, 1, R * cin)),
         "lift_b": np.zeros(width)}
    for b in range(nblocks):
        for j in (0, 1):
            p["b%d_w%d" % (b, j)] = rng.normal(0, np.sqrt(2.0 / (K5 * width)), (width, K5, width))
            p["b%d_b%d" % (b, j)] = np.zeros(width)
    p["head_w"] = rng.normal(0, np.sqrt(1.0 / width), (R * cout, 1, width))
    p["head_b"] = np.zeros(R * cout)
    return p


def conv(x, W, b, rnd=_ident):
    """x (N, L, Ci), W (Co, k, Ci), b (Co) -> (N, L, Co), zero padding."""
    x, W = rnd(x), rnd(W)
    N, L, Ci = x.shape
    Co, k, _ = W.shape
    c = (k - 1) // 2
    y = np.broadcast_to(b, (N, L, Co)).astype(np.float64).copy()
    for t in range(k):
        s = t - c
        xs = np.zeros_like(x)
        if s >= 0:
            xs[:, :L - s] = x[:, s:] if s < L else 0
        else:
            xs[:, -s:] = x[:, :L + s] if -s < L else 0
        y += np.einsum("nli,oi->nlo", xs, W[:, t, :])
    return y


def conv_backward(x, W, dy, rnd=_ident):
    """Gradients of conv: returns dx, dW, db (db from the unrounded dy)."""
    db = dy.sum(axis=(0, 1))
    x, W, dy = rnd(x), rnd(W), rnd(dy)
    N, L, Ci = x.shape
    Co, k, _ = W.shape
    c = (k - 1) // 2
    dx = np.zeros_like(x)
    dW = np.zeros_like(W)
    for t in range(k):
        s = t - c
        xs = np.zeros_like(x)
        if s >= 0:
            xs[:, :L - s] = x[:, s:] if s < L else 0
        else:
            xs[:, -s:] = x[:, :L + s] if -s < L else 0
        dW[:, t, :] = np.einsum("nlo,nli->oi", dy, xs)
        g = np.einsum("nlo,oi->nli", dy, W[:, t, :])  # gradient wrt xs
        if s >= 0:
            if s < L:
                dx[:, s:] += g[:, :L - s]
        else:
            if -s < L:
                dx[:, :L + s] += g[:, -s:]
    return dx, dW, db


def unshuffle(x):
    N, L, C = x.shape
    return x.reshape(N, L // R, R * C)


def shuffle(y, cout):
    N, Lq, _ = y.shape
    return y.reshape(N, Lq * R, cout)


def forward(p, x, nblocks, cout, rnd=_ident):
    """x (N, L, Cin) -> (N, L, Cout); returns (out, cache)."""
    cache = {}
    h = conv(unshuffle(x), p["lift_w"], p["lift_b"], rnd)
    cache["x0"] = unshuffle(x)
    for b in range(nblocks):
        a0 = np.maximum(h, 0.0)
        z0 = conv(a0, p["b%d_w0" % b], p["b%d_b0" % b], rnd)
        a1 = np.maximum(z0, 0.0)
        z1 = conv(a1, p["b%d_w1" % b], p["b%d_b1" % b], rnd)
        cache[b] = (h, a0, z0, a1)
        h = h + z1
    a = np.maximum(h, 0.0)
    cache["head_in"] = (h, a)
    y = conv(a, p["head_w"], p["head_b"], rnd)
    return shuffle(y, cout), cache


def loss_and_grad(p, x, target, mask, nblocks, cout, rnd=_ident):
    """Masked mean-squared error L = sum(mask (y - target)^2) / sum(mask * cout)
    and its gradient wrt every parameter. mask (N, L)."""
    y, cache = forward(p, x, nblocks, cout, rnd)
    norm = mask.sum() * cout
    diff = (y - target) * mask[..., None]
    loss = float((diff * (y - target)).sum() / norm)
    dy = 2.0 * diff / norm
    g = {}
    dyq = unshuffle(dy)
    h, a = cache["head_in"]
    da, g["head_w"], g["head_b"] = conv_backward(a, p["head_w"], dyq, rnd)
    dh = da * (h > 0)
    for b in reversed(range(nblocks)):
        hb, a0, z0, a1 = cache[b]
        da1, g["b%d_w1" % b], g["b%d_b1" % b] = conv_backward(a1, p["b%d_w1" % b], dh, rnd)
        dz0 = da1 * (z0 > 0)
        da0, g["b%d_w0" % b], g["b%d_b0" % b] = conv_backward(a0, p["b%d_w0" % b], dz0, rnd)
        dh = dh + da0 * (hb > 0)
    _, g["lift_w"], g["lift_b"] = conv_backward(cache["x0"], p["lift_w"], dh, rnd)
    return loss, g, y


def flatten(p, nblocks):
    """Parameter dict -> one vector in the layer order lift, b0 w0, b0 w1, ...,
    head; per layer the weights W[o][t][i] then the biases."""
    keys = [("lift_w", "lift_b")]
    for b in range(nblocks):
        keys += [("b%d_w0" % b, "b%d_b0" % b), ("b%d_w1" % b, "b%d_b1" % b)]
    keys.append(("head_w", "head_b"))
    return np.concatenate([np.concatenate([p[w].reshape(-1), p[bb].reshape(-1)]) for w, bb in keys])


def unflatten(v, cin, cout, width, nblocks):
    """Inverse of flatten for the shapes of init_params."""
    shapes = init_params(cin, cout, width, nblocks)
    keys = ["lift_w", "lift_b"]
    for b in range(nblocks):
        keys += ["b%d_w0" % b, "b%d_b0" % b, "b%d_w1" % b, "b%d_b1" % b]
    keys += ["head_w", "head_b"]
    out, off = {}, 0
    for k in keys:
        n = shapes[k].size
        out[k] = np.asarray(v[off:off + n], dtype=np.float64).reshape(shapes[k].shape)
        off += n
    assert off == len(v)
    return out


def adam(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, Algorithm 1, with bias correction) on the
    dicts p (updated in place), m and v (moment estimates, updated in place);
    ``step`` counts from 1."""
    c1, c2 = 1.0 - beta1 ** step, 1.0 - beta2 ** step
    for k in p:
        m[k] = beta1 * m[k] + (1.0 - beta1) * g[k]
        v[k] = beta2 * v[k] + (1.0 - beta2) * g[k] ** 2
        p[k] = p[k] - lr * (m[k] / c1) / (np.sqrt(v[k] / c2) + eps)
    return p


# ---- moment blocks, network inputs and the conservative update ---------------
# A tube of nx cells per sublattice has 2 nx points; point (s, x) has index
# s nx + x and fine position 2x + s. A moment block is [4][2 nx]: rho, u_x,
# theta_T, E_R. Conserved densities U = (rho, rho u_x, E, E_R) with
# E = rho u_x^2 / 2 + 3 rho theta_T / 2 + E_R (translational energy of three
# degrees of freedom plus the rotational energy density).

def conserved(v):
    """v (4, ...) = (rho, u_x, theta_T, E_R) -> U (4, ...)."""
    rho, ux, th, er = v
    return np.stack([rho, rho * ux, 0.5 * rho * ux ** 2 + 1.5 * rho * th + er, er])


def primitive(U):
    """Inverse of conserved."""
    rho, m, E, er = U
    ux = m / rho
    return np.stack([rho, ux, (E - 0.5 * m * ux - er) / (1.5 * rho), er])


def position_order(block, nx):
    """[4][2 nx] in point order -> [4][2 nx] in fine-position order 2x + s."""
    out = np.empty_like(block)
    out[:, 0::2] = block[:, :nx]
    out[:, 1::2] = block[:, nx:]
    return out


def point_order(seq, nx):
    """Inverse of position_order."""
    out = np.empty_like(seq)
    out[:, :nx] = seq[:, 0::2]
    out[:, nx:] = seq[:, 1::2]
    return out


_M64 = (1 << 64) - 1


def splitmix64(seed, n):
    """Output n + 1 of SplitMix64 seeded with ``seed`` (Steele, Lea & Flood,
    "Fast splittable pseudorandom number generators", OOPSLA 2014): add the
    golden gamma 0x9E3779B97F4A7C15 n + 1 times, then the output mix
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB;
    z ^= z >> 31 (all modulo 2^64)."""
    z = (seed + (n + 1) * 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def pack(src, tgt, nx, res, cond, pad, crop, length, margin, shift, scale, out_scale,
         prev=None, dscale=(1.0, 1.0, 1.0, 1.0), noise=None, seed=0, seq_index=0):
    """Network input x (length, 11) of one padded tube, and (when tgt is not
    None) the normalised target increments (length, 4) and the loss mask
    (length,). Features: (v - shift) / scale, (v - v_prev) / dscale (zero
    without a previous block and in the padding), cond, inside indicator.
    res (2, 4): left / right reservoir (rho, u_x, theta_T, E_R). ``noise``: at
    tube points v_k is replaced by v_k + noise_k sqrt(3) (2 u - 1) with u =
    2^-53 (splitmix64(seed, ((seq_index << 32) | l) 4 + k) >> 11), and
    features and targets use the perturbed state."""
    shift, scale = np.asarray(shift, np.float32), np.asarray(scale, np.float32)
    dscale = np.asarray(dscale, np.float32)
    s = position_order(np.asarray(src, np.float64), nx)
    q = position_order(np.asarray(prev, np.float64), nx) if prev is not None else None
    t = position_order(np.asarray(tgt, np.float64), nx) if tgt is not None else None
    x = np.zeros((length, 11), np.float32)
    target = np.zeros((length, 4))
    mask = np.zeros(length)
    for l in range(length):
        p = crop + l - pad
        inside = 0 <= p < 2 * nx
        v = s[:, p].copy() if inside else np.asarray(res[0 if p < 0 else 1], np.float64)
        if inside and noise is not None:
            for k in range(4):
                if noise[k] != 0.0:
                    h = splitmix64(seed, (((seq_index << 32) | l) * 4 + k) & _M64)
                    u = (h >> 11) * 2.0 ** -53
                    v[k] += float(np.float32(noise[k])) * 1.7320508075688772 * (2.0 * u - 1.0)
        w = q[:, p] if (inside and prev is not None) else v
        x[l, :4] = (v.astype(np.float32) - shift) / scale
        x[l, 4:8] = (v.astype(np.float32) - w.astype(np.float32)) / dscale
        x[l, 8:10] = cond
        x[l, 10] = 1.0 if inside else 0.0
        if t is not None and inside and margin <= l < length - margin:
            target[l] = (conserved(t[:, p]) - conserved(v)) / np.asarray(out_scale, np.float64)
            mask[l] = 1.0
    return x, target, mask


def apply(block, y, nx, pad, crop, out_scale, project):
    """Moment block after one network application: increments out_scale * y at
    the tube's positions (y (length, 4) of its sequence); with ``project`` the
    mass and energy increments d are replaced by d - |d| sum(d) / sum(|d|)
    (zero net change, the correction put where the change is). Returns
    (new block, invalid, (sum rho, sum E))."""
    v = position_order(np.asarray(block, np.float64), nx)
    d = (np.asarray(y, np.float64)[pad - crop:pad - crop + 2 * nx] * np.asarray(out_scale, np.float64)).T
    if project:
        for k in (0, 2):
            a = np.abs(d[k]).sum()
            if a > 0:
                d[k] = d[k] - np.abs(d[k]) * (d[k].sum() / a)
    U = conserved(v) + d
    w = primitive(U)
    bad = bool(np.any(~np.isfinite(w)) or np.any(w[0] <= 0) or np.any(w[2] <= 0) or np.any(w[3] <= 0))
    return point_order(w, nx), bad, (float(U[0].sum()), float(U[2].sum()))
