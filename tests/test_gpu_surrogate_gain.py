"""What the trained surrogate gains over the method without it.

The surrogate's network (width 128, 6 residual blocks, 0.99 M parameters) is
trained on the GPU by the library's own forward, backward and Adam kernels
(6000 Adam steps of 32 crops) on the batched LBM's snapshots of 96 tubes of
the shock-tube sweep (lengths 300-800 cells), then evaluated on 24 held-out
tubes of another seed:

1. One window (32 steps) from the LBM's own state, every window of every tube
   (the rollout with a spot check in every window records the network's
   relative L1 density error against the LBM's 32 steps): the trained network
   against the method without a network, i.e. leaving the state unchanged for
   32 steps (a zero network), and against the same network untrained.
2. The rollout with spot checks every fourth window, hand-over from the last
   accepted state, accumulated-error bound 1%: LBM steps run (spot checks and
   remainders) against the plain LBM's steps, and the final relative L1 density
   error of each tube against the plain LBM. The zero network is handed to the
   LBM at its first spot check and saves nothing.

Measured on GB300: one-window median error 0.18% trained, 1.2% untrained,
3.5% without a network; the rollout ran 0.65 (every 4th window checked) and
0.73 (every 2nd) of the plain LBM's steps with final errors of median 0.52% /
0.56%, max 2.6%, where the zero network saves nothing. The bars below leave
about a factor of two.
"""
import numpy as np
import pytest

import paper_2201_05280_gb300 as rpk
from paper_2201_05280_gb300 import surrogate as SG
import rpk_inputs as I

pytestmark = pytest.mark.gpu

T0 = 0.2948964908710633
TRAIN_STEPS = 6000
WIDTH, BLOCKS = 128, 6


@pytest.fixture(scope="module")
def trained():
    from paper_2201_05280_gb300 import build as B
    B.build()
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    specs, f = I.tube_sweep(96, T0, seed=71, L=(300, 800))
    tubes, cond = SG.make_tubes(specs, f, T0)
    data = SG.TrainingSet(tubes, cond, f, diffusion="implicit")
    cfg = SG.default_config(T0)
    net = rpk.Net(SG.CIN, SG.COUT, WIDTH, BLOCKS, seed=5)
    untrained = rpk.Net(SG.CIN, SG.COUT, WIDTH, BLOCKS, seed=5)
    hist = SG.train(net, cfg, data, TRAIN_STEPS, batch=32, crop_len=512,
                    noise=[3e-4, 3e-4, 1e-4, 1e-4], seed=5)
    torch.cuda.synchronize()
    del data
    specs, f = I.tube_sweep(24, T0, seed=72, L=(300, 800))
    etubes, econd = SG.make_tubes(specs, f, T0)
    blk0 = SG.initial_blocks(etubes, f)
    return net, untrained, etubes, econd, blk0, hist


def _zero_net():
    net = rpk.Net(SG.CIN, SG.COUT, WIDTH, BLOCKS, seed=5)
    net.set_params(np.zeros(net.num_params, dtype=np.float32))
    return net


def _window_errors(net, tubes, cond, blk0):
    cfg = SG.default_config(T0, spot_every=1, l1_tol=1e300, drift_tol=1e300, anchor=1,
                            lbm_diffusion=1)
    R = rpk.Rollout(net, cfg, tubes, cond)
    R.run(blk0.clone())
    e = R.errors()
    R.close()
    return e[np.isfinite(e)]


def _plain_lbm(tubes, blk0):
    B = rpk.Batch(tubes, precision="f32", save_every=1 << 30)
    B.set_diffusion("implicit")
    B.init_device(blk0).run()
    out = B.moments_device().cpu().numpy()
    offs = B.block_offsets
    B.close()
    return out, offs


def test_one_window_error_beats_the_method_without_a_network(trained):
    net, untrained, tubes, cond, blk0, hist = trained
    zero = _zero_net()
    e_tr = _window_errors(net, tubes, cond, blk0)
    e_un = _window_errors(untrained, tubes, cond, blk0)
    e_0 = _window_errors(zero, tubes, cond, blk0)
    zero.close()
    med = {k: float(np.median(v)) for k, v in (("trained", e_tr), ("untrained", e_un), ("no network", e_0))}
    print("one-window relative L1 density error, median over %d windows: %s; trained p90 %.2e; "
          "training loss %.3e -> %.3e" % (e_tr.size, med, np.percentile(e_tr, 90),
                                          np.mean(hist[:20]), np.mean(hist[-100:])))
    assert e_tr.size == e_0.size > 50
    assert med["trained"] <= 5e-3
    assert med["trained"] <= 0.2 * med["no network"]
    assert med["trained"] <= 0.3 * med["untrained"]


@pytest.mark.parametrize("spot_every,l1_tol", [(4, 1e-2), (2, 1e-2)])
def test_rollout_saves_lbm_steps(trained, spot_every, l1_tol):
    net, untrained, tubes, cond, blk0, hist = trained
    ref, offs = _plain_lbm(tubes, blk0)
    plain_steps = int(sum(t["nsteps"] for t in tubes))
    res = {}
    for name, n in (("trained", net), ("no network", _zero_net())):
        cfg = SG.default_config(T0, spot_every=spot_every, l1_tol=l1_tol, anchor=1, lbm_diffusion=1)
        R = rpk.Rollout(n, cfg, tubes, cond)
        st = blk0.clone()
        s = R.run(st)
        R.close()
        got = st.cpu().numpy()
        lbm = int((s["checks"] * cfg.jump + s["lbm_steps"]).sum())
        l1 = np.array([np.abs(got[o:o + 2 * t["nx"]] - ref[o:o + 2 * t["nx"]]).sum() /
                       np.abs(ref[o:o + 2 * t["nx"]]).sum() for o, t in zip(offs, tubes)])
        res[name] = (lbm / plain_steps, float(np.median(l1)), float(l1.max()), int(s["windows"].sum()))
        if name == "no network":
            n.close()
    print("spot every %d, l1_tol %g: LBM steps / plain LBM steps, median and max final L1 vs plain "
          "LBM, network windows kept: %s" % (spot_every, l1_tol, res))
    assert res["no network"][0] >= 1.0 and res["no network"][3] == 0
    # the trained network saves LBM steps at a median final error below 1%
    assert res["trained"][0] <= 0.85
    assert res["trained"][3] > 0
    assert res["trained"][1] <= 1e-2
    assert res["trained"][2] <= 5e-2
