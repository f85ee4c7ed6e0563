"""GPU checks of the surrogate pipeline around the network: input/target
packing and the conservative update against the oracle's definitions, the
batch's device-side initialisation and moments, and the rollout engine's
hand-over logic (drift, spot checks, fallback) against explicit compositions of
batched LBM runs.

Packing: features are one float32 subtraction and division (bitwise equal up
to one rounding); targets and updates are evaluated in FP64 and rounded to
float32 (relative 1e-6). The rollout's LBM pieces start from the same moment
blocks as the composed reference runs, so those comparisons are bitwise."""
import numpy as np
import pytest

from oracle import surrogate as S
from oracle import params as PM
import paper_2201_05280_gb300 as rpk
import rpk_inputs as I

pytestmark = pytest.mark.gpu

T0 = 0.2948964908710633
CS = np.sqrt(1.4 * T0)
JUMP = 32


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    from paper_2201_05280_gb300 import build as B
    B.build()
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


def _tubes(n, L, seed, min_steps=0):
    specs, f = I.tube_sweep(n, T0, seed=seed, L=L)
    tubes = []
    for i, sp in enumerate(specs):
        lo, hi = 2 * sum(s["nx"] for s in specs[:i]), 2 * sum(s["nx"] for s in specs[:i + 1])
        nu = sp["kn"] * CS * sp["nx"]
        eta, etaB, kap = PM.gas_from_nondim(1.4, nu, sp["lam"], sp["pr"])
        d, tau, tau1, b, kr = PM.relax_from_gas(1.4, eta, etaB, kap, 0.0)
        thmax = max(float(np.max((3 * f["T"][lo:hi] + d * f["R"][lo:hi]) / (3 + d))),
                    float(np.max((3 * sp["res"][[4, 10]] + d * sp["res"][[5, 11]]) / (3 + d))))
        relax = dict(delta=d, tau=tau, tau1=tau1, b=b, k_r=kr, nsub=PM.nsub_for(d, tau, tau1, kr, thmax, 1))
        tubes.append({"nx": sp["nx"], "nsteps": max(sp["nsteps"], min_steps), "relax": relax,
                      "res": sp["res"], "lo": lo, "hi": hi, "cond": (np.log(nu), sp["lam"])})
    return tubes, f


def _blocks(tubes, f):
    """Initial moment blocks through the library (the LBM's own moments of its
    initial state) as a CUDA tensor."""
    B = rpk.Batch(tubes, precision="f32", save_every=1 << 20)
    B.init_fields(f["rho"], f["u"], f["T"], f["R"])
    out = B.moments_device()
    B.close()
    return out


def _res4(t):
    r = t["res"]
    d = t["relax"]["delta"]
    return np.array([[r[0], r[1], r[4], 0.5 * d * r[0] * r[5]], [r[6], r[7], r[10], 0.5 * d * r[6] * r[11]]])


def test_device_blocks_match_fields_and_reinitialise():
    import torch
    tubes, f = _tubes(4, (30, 90), seed=21)
    blk = _blocks(tubes, f).cpu().numpy()
    off = 0
    for t in tubes:
        lo, hi = t["lo"], t["hi"]
        np2 = hi - lo
        ref = np.stack([f["rho"][lo:hi], f["u"][0, lo:hi], f["T"][lo:hi],
                        0.5 * t["relax"]["delta"] * f["rho"][lo:hi] * f["R"][lo:hi]])
        got = blk[off:off + 4 * np2].reshape(4, np2)
        np.testing.assert_allclose(got, ref, rtol=2e-6, atol=2e-7)
        off += 4 * np2
    # device initialisation from the blocks reproduces them; step counts patch the run
    A = rpk.Batch(tubes, precision="f32", save_every=1 << 20)
    A.init_device(torch.tensor(blk, device="cuda"))
    np.testing.assert_allclose(A.moments_device().cpu().numpy(), blk, rtol=2e-6, atol=2e-7)
    short = [dict(t, nsteps=min(t["nsteps"], 20)) for t in tubes]
    Bs = rpk.Batch(short, precision="f32", save_every=1 << 20)
    Bs.init_device(torch.tensor(blk, device="cuda")).run()
    A.set_steps([t["nsteps"] for t in short]).run()
    np.testing.assert_array_equal(A.moments_device().cpu().numpy(), Bs.moments_device().cpu().numpy())
    with pytest.raises(rpk.RpkError):
        A.set_steps([t["nsteps"] + 1 for t in tubes])
    A.close()
    Bs.close()


def _cfg(**kw):
    base = dict(jump=JUMP, pad=16, spot_every=0, project=0, drift_tol=1e300, l1_tol=1e300,
                in_shift=(0.5, 0.0, T0, 0.15), in_scale=(0.3, 0.3, 0.1, 0.1),
                out_scale=(0.02, 0.01, 0.03, 0.01), in_dscale=(0.01, 0.02, 0.004, 0.005))
    base.update(kw)
    return rpk.SurConfig.make(**base)


def test_pack_matches_oracle():
    import torch
    rng = np.random.default_rng(22)
    cfg = _cfg()
    nxs = [7, 20, 13]
    blocks = [np.stack([rng.uniform(0.2, 1, 2 * n), rng.normal(0, 0.2, 2 * n), rng.uniform(0.15, 0.4, 2 * n),
                        rng.uniform(0.05, 0.4, 2 * n)]) for n in nxs]
    tgts = [b * rng.uniform(0.9, 1.1, b.shape) for b in blocks]
    prevs = [b * rng.uniform(0.95, 1.05, b.shape) for b in blocks]
    store = np.concatenate([b.ravel() for b in blocks] + [b.ravel() for b in tgts] +
                           [b.ravel() for b in prevs]).astype(np.float32)
    offs = np.cumsum([0] + [8 * n for n in nxs])
    toff = offs[-1]
    seqs, refs = [], []
    out = 0
    for i, (n, crop, length, margin) in enumerate(zip(nxs, [0, 10, 3], [48, 36, 60], [0, 4, 4])):
        res = rng.uniform(0.1, 1.0, (2, 4))
        cond = rng.normal(size=2)
        prev = 2 * toff + offs[i] if i != 1 else -1  # the middle sequence has no previous window
        seqs.append(dict(src=offs[i], tgt=toff + offs[i], prev=prev, out=out, nx=n, len=length, crop=crop,
                         res=res, cond=cond))
        refs.append(S.pack(blocks[i].astype(np.float32).astype(np.float64),
                           tgts[i].astype(np.float32).astype(np.float64), n, res.astype(np.float32),
                           cond.astype(np.float32), cfg.pad, crop, length, margin, list(cfg.in_shift),
                           list(cfg.in_scale), list(cfg.out_scale),
                           prev=prevs[i].astype(np.float32).astype(np.float64) if i != 1 else None,
                           dscale=list(cfg.in_dscale)) + (margin,))
        out += length
    for i, sq in enumerate(seqs):
        x, t, m = rpk.sur_pack(cfg, torch.tensor(store, device="cuda"), [sq], margin=refs[i][3])
        sl = slice(sq["out"], sq["out"] + sq["len"])
        np.testing.assert_allclose(x.cpu().numpy()[sl], refs[i][0], rtol=2.4e-7, atol=1e-30)
        np.testing.assert_array_equal(m.cpu().numpy()[sl], refs[i][2])
        np.testing.assert_allclose(t.cpu().numpy()[sl], refs[i][1], rtol=1e-6, atol=1e-6)
    # perturbed sources: all sequences in one call (sequence index = draw stream)
    noise = (1e-3, 2e-3, 5e-4, 5e-4)
    x, t, m = rpk.sur_pack(cfg, torch.tensor(store, device="cuda"), seqs, margin=0, noise=noise, seed=99)
    for i, sq in enumerate(seqs):
        ref = S.pack(blocks[i].astype(np.float32).astype(np.float64),
                     tgts[i].astype(np.float32).astype(np.float64), nxs[i], sq["res"].astype(np.float32),
                     np.asarray(sq["cond"], np.float32), cfg.pad, sq["crop"], sq["len"], 0,
                     list(cfg.in_shift), list(cfg.in_scale), list(cfg.out_scale),
                     prev=prevs[i].astype(np.float32).astype(np.float64) if i != 1 else None,
                     dscale=list(cfg.in_dscale), noise=noise, seed=99, seq_index=i)
        sl = slice(sq["out"], sq["out"] + sq["len"])
        np.testing.assert_allclose(x.cpu().numpy()[sl], ref[0], rtol=1e-6, atol=1e-6)
        np.testing.assert_allclose(t.cpu().numpy()[sl], ref[1], rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("project", [0, 1])
def test_apply_matches_oracle(project):
    import torch
    rng = np.random.default_rng(23 + project)
    cfg = _cfg(project=project, pad=8)
    nxs = [9, 31, 4]
    blocks = [np.stack([rng.uniform(0.2, 1, 2 * n), rng.normal(0, 0.2, 2 * n), rng.uniform(0.15, 0.4, 2 * n),
                        rng.uniform(0.05, 0.4, 2 * n)]).astype(np.float32) for n in nxs]
    state = np.concatenate([b.ravel() for b in blocks])
    offs = np.cumsum([0] + [8 * n for n in nxs])
    lens = [2 * n + 16 for n in nxs]
    lens = [(L + 3) // 4 * 4 for L in lens]
    youts = np.cumsum([0] + lens)
    y = rng.normal(0, 1, (youts[-1], 4)).astype(np.float32)
    seqs = [dict(src=offs[i], out=youts[i], nx=n, len=lens[i], res=np.ones((2, 4)), cond=(0, 0))
            for i, n in enumerate(nxs)]
    nxt, flags, tot = rpk.sur_apply(cfg, torch.tensor(state, device="cuda"), torch.tensor(y, device="cuda"), seqs)
    nxt = nxt.cpu().numpy()
    for i, n in enumerate(nxs):
        ref, bad, rt = S.apply(blocks[i].astype(np.float64), y[youts[i]:youts[i + 1]].astype(np.float64), n,
                               cfg.pad, 0, list(cfg.out_scale), project)
        got = nxt[offs[i]:offs[i + 1]].reshape(4, 2 * n)
        assert flags[i] == int(bad)
        if not bad:
            np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(tot[i], rt, rtol=1e-10)


def _net(head_bias=None):
    net = rpk.Net(11, 4, 16, 0, seed=1)
    v = np.zeros(net.num_params, dtype=np.float32)
    if head_bias is not None:
        v[-16:] = head_bias
    net.set_params(v)
    return net


def _lbm(tubes, blk, steps, only=None):
    """Composed reference: one batched LBM run of `steps` from the blocks; the
    tubes in `only` (default: those with steps > 0) take the LBM's moments."""
    import torch
    B = rpk.Batch(tubes, precision="f32", save_every=1 << 20)
    B.init_device(blk).set_steps(steps).run()
    m = B.moments_device()
    out = blk.clone()
    offs = B.block_offsets
    for i, t in enumerate(tubes):
        if (only is None and steps[i] > 0) or (only is not None and i in only):
            out[offs[i]:offs[i] + 8 * t["nx"]] = m[offs[i]:offs[i] + 8 * t["nx"]]
    B.close()
    torch.cuda.synchronize()
    return out


def test_rollout_zero_network_keeps_state_then_lbm_remainder():
    tubes, f = _tubes(5, (40, 120), seed=24, min_steps=70)
    blk = _blocks(tubes, f)
    net = _net()
    R = rpk.Rollout(net, _cfg(), tubes, [t["cond"] for t in tubes])
    state = blk.clone()
    st = R.run(state)
    J = [t["nsteps"] // JUMP for t in tubes]
    np.testing.assert_array_equal(st["windows"], J)
    np.testing.assert_array_equal(st["fail_step"], -1)
    ref = _lbm(tubes, blk, [t["nsteps"] - JUMP * j for t, j in zip(tubes, J)])
    np.testing.assert_array_equal(state.cpu().numpy(), ref.cpu().numpy())
    R.close()


def test_rollout_spot_every_window_is_the_restarted_lbm():
    tubes, f = _tubes(4, (40, 100), seed=25, min_steps=70)
    blk = _blocks(tubes, f)
    net = _net()
    R = rpk.Rollout(net, _cfg(spot_every=1), tubes, [t["cond"] for t in tubes])
    state = blk.clone()
    st = R.run(state)
    J = [t["nsteps"] // JUMP for t in tubes]
    np.testing.assert_array_equal(st["checks"], J)
    np.testing.assert_array_equal(st["windows"], 0)
    ref = blk.clone()
    for w in range(max(J)):
        act = [i for i in range(len(tubes)) if w < J[i]]
        ref = _lbm(tubes, ref, [JUMP if i in act else 0 for i in range(len(tubes))], only=act)
    ref = _lbm(tubes, ref, [t["nsteps"] - JUMP * j for t, j in zip(tubes, J)])
    np.testing.assert_array_equal(state.cpu().numpy(), ref.cpu().numpy())
    R.close()


def test_rollout_l1_bound_hands_tubes_to_the_lbm():
    tubes, f = _tubes(4, (40, 100), seed=26, min_steps=100)
    blk = _blocks(tubes, f)
    net = _net()
    R = rpk.Rollout(net, _cfg(spot_every=4, l1_tol=0.0), tubes, [t["cond"] for t in tubes])
    state = blk.clone()
    st = R.run(state)
    # the zero network misses the first window's change: every tube is handed
    # over after the LBM's first (spot-check) window
    np.testing.assert_array_equal(st["fail_step"], JUMP)
    assert np.all(st["est"] > 0)
    ref = _lbm(tubes, blk, [JUMP] * len(tubes))
    ref = _lbm(tubes, ref, [t["nsteps"] - JUMP for t in tubes])
    np.testing.assert_array_equal(state.cpu().numpy(), ref.cpu().numpy())
    R.close()


def test_rollout_drift_check_and_projection():
    tubes, f = _tubes(3, (40, 100), seed=27, min_steps=70)
    blk = _blocks(tubes, f)
    bias = np.zeros(16, dtype=np.float32)
    bias[0::4] = 1.0  # a uniform mass increment of out_scale[0] per point and window
    net = _net(bias)
    # without projection the mass drift is about 2e-2 of the tube's mass: the LBM runs everything
    R = rpk.Rollout(net, _cfg(drift_tol=1e-4), tubes, [t["cond"] for t in tubes])
    state = blk.clone()
    st = R.run(state)
    np.testing.assert_array_equal(st["fail_step"], 0)
    np.testing.assert_array_equal(st["windows"], 0)
    ref = _lbm(tubes, blk, [t["nsteps"] for t in tubes])
    np.testing.assert_array_equal(state.cpu().numpy(), ref.cpu().numpy())
    R.close()
    # the projection removes a uniform increment entirely: the state is kept
    R = rpk.Rollout(net, _cfg(drift_tol=1e-4, project=1), tubes, [t["cond"] for t in tubes])
    state = blk.clone()
    st = R.run(state)
    np.testing.assert_array_equal(st["fail_step"], -1)
    J = [t["nsteps"] // JUMP for t in tubes]
    np.testing.assert_array_equal(st["windows"], J)
    ref = _lbm(tubes, blk, [t["nsteps"] - JUMP * j for t, j in zip(tubes, J)])
    np.testing.assert_array_equal(state.cpu().numpy(), ref.cpu().numpy())
    R.close()


def test_rollout_without_anchor_reruns_handed_tubes_from_the_start():
    tubes, f = _tubes(4, (40, 100), seed=28, min_steps=100)
    blk = _blocks(tubes, f)
    net = _net()
    R = rpk.Rollout(net, _cfg(spot_every=4, l1_tol=0.0, anchor=0), tubes, [t["cond"] for t in tubes])
    state = blk.clone()
    st = R.run(state)
    np.testing.assert_array_equal(st["fail_step"], 0)
    np.testing.assert_array_equal(st["checks"], 1)
    np.testing.assert_array_equal(st["lbm_steps"], [t["nsteps"] for t in tubes])
    ref = _lbm(tubes, blk, [t["nsteps"] for t in tubes])
    np.testing.assert_array_equal(state.cpu().numpy(), ref.cpu().numpy())
    # with a generous bound the zero network's windows are all kept
    R2 = rpk.Rollout(net, _cfg(spot_every=4, l1_tol=10.0, anchor=0), tubes, [t["cond"] for t in tubes])
    state = blk.clone()
    st = R2.run(state)
    J = [t["nsteps"] // JUMP for t in tubes]
    np.testing.assert_array_equal(st["windows"], J)
    np.testing.assert_array_equal(st["fail_step"], -1)
    R.close()
    R2.close()
