"""Learned surrogate of the batched shock tubes: training data from the batched
LBM, the training loop and the rollout set-up. Orchestration only: the LBM,
input packing, the network's forward and backward passes, Adam and the
conservative update all run in librpk's kernels (see ``Net``, ``sur_pack``,
``Rollout``); this module draws minibatches and marshals descriptors.

A training pair is (moments at step 32 k, moments at step 32 (k + 1)) of one
tube, with the moments at step 32 (k - 1) as the previous window (none for
k = 0); the network sees a crop of the tube padded with its reservoir states
and learns the increments of the conserved densities (rho, rho u_x, E, E_R)
over the window. The paper has no learned component; the data come from its
method."""
import math

import numpy as np

import paper_2201_05280_gb300 as rpk

GAMMA = 1.4
PR = 0.71
CIN, COUT = 11, 4

# numpy view of rpk_sur_seq (88 bytes)
SEQ_DTYPE = np.dtype([("src", "<i8"), ("tgt", "<i8"), ("prev", "<i8"), ("out", "<i8"),
                      ("nx", "<i4"), ("len", "<i4"), ("crop", "<i4"), ("pad_", "<i4"),
                      ("res", "<f4", (2, 4)), ("cond", "<f4", (2,))])
assert SEQ_DTYPE.itemsize == 88

# Feature and output scales for the sweep's states (left state rho = 1,
# theta = theta0; right states down to rho ~ 0.12, theta ~ 0.42 theta0; flows
# up to |u| ~ 0.6 c_s). Output scales are the typical size of a window's
# increments of rho, rho u_x, E and E_R near the waves.
def default_config(theta0, **kw):
    base = dict(jump=32, pad=128, spot_every=8, project=1, drift_tol=1e-4, l1_tol=1e-2,
                in_shift=(0.55, 0.0, theta0, 0.17), in_scale=(0.3, 0.3, 0.1, 0.1),
                out_scale=(0.015, 0.011, 0.013, 0.0045), in_dscale=(0.015, 0.02, 0.005, 0.005))
    base.update(kw)
    return rpk.SurConfig.make(**base)


def cond_features(nu, lam):
    """Conditioning of a tube: lattice kinematic viscosity nu (log) and
    eta_B / eta, centred on the sweep's ranges."""
    return ((math.log(nu) - 2.2) / 1.7, (lam - 1.15) / 0.5)


def make_tubes(specs, fields, theta0):
    """Sweep specs (rpk_inputs.tube_sweep) -> tube dicts with raw relaxation
    parameters from the library's gas mapping and explicit FTCS sub-step
    counts (rpk_auto_nsub on the tube's hottest initial state), and the
    conditioning features (ntubes, 2)."""
    cs = rpk.sound_speed(GAMMA)
    tubes, cond = [], []
    off = 0
    for sp in specs:
        nu = sp["kn"] * cs * sp["nx"]  # Kn = nu / (c_s L), L = cells along the tube
        eta, etaB, kap = rpk.gas_from_nondim(GAMMA, nu, sp["lam"], sp.get("pr", PR))
        r = rpk.map_gas(GAMMA, eta, etaB, kap, 0.0)
        sl = slice(off, off + 2 * sp["nx"])
        r["nsub"] = rpk.auto_nsub_fields(r, fields["T"][sl], fields["R"][sl], sp["res"], 1)
        tubes.append({"nx": sp["nx"], "nsteps": sp["nsteps"], "relax": r, "res": sp["res"]})
        cond.append(cond_features(nu, sp["lam"]))
        off += 2 * sp["nx"]
    return tubes, np.asarray(cond, dtype=np.float32)


def reservoirs(tube):
    """(2, 4) reservoir states (rho, u_x, theta_T, E_R) of a tube dict."""
    return rpk.tube_reservoirs(tube)


class TrainingSet:
    """Snapshots of an LBM run of the tubes held on the device, with the index
    of all consecutive pairs."""

    def __init__(self, tubes, cond, fields, save_every=32, diffusion="ftcs", stream=None):
        import torch
        bt = rpk.Batch(tubes, precision="f32", save_every=save_every, stream=stream)
        bt.set_diffusion(diffusion)
        bt.init_fields(fields["rho"], fields["u"], fields["T"], fields["R"])
        self.tune = bt.autotune()
        bt.run()
        torch.cuda.synchronize()
        snaps = bt.snapshots()
        bt.close()
        self.tubes, self.cond = tubes, np.asarray(cond, np.float32)
        self.res = np.stack([reservoirs(t) for t in tubes])
        offs, src, tgt, prev, tube_of = 0, [], [], [], []
        flat = []
        for i, s in enumerate(snaps):
            n = s.shape[0]
            blk = 4 * s.shape[2]
            for k in range(n - 1):
                src.append(offs + k * blk)
                tgt.append(offs + (k + 1) * blk)
                prev.append(offs + (k - 1) * blk if k > 0 else -1)
                tube_of.append(i)
            flat.append(s.reshape(-1))
            offs += n * blk
        self.store = torch.from_numpy(np.concatenate(flat)).cuda()
        self.src = np.asarray(src, np.int64)
        self.tgt = np.asarray(tgt, np.int64)
        self.prev = np.asarray(prev, np.int64)
        self.tube = np.asarray(tube_of, np.int64)
        self.nx = np.array([t["nx"] for t in tubes], np.int32)

    def __len__(self):
        return len(self.src)

    def descriptors(self, idx, crop_len, pad, rng):
        """Sequence descriptors of pairs idx, each a random crop of crop_len
        points of the padded tube."""
        n = len(idx)
        d = np.zeros(n, SEQ_DTYPE)
        tb = self.tube[idx]
        nx = self.nx[tb]
        full = 2 * nx + 2 * pad
        d["src"], d["tgt"], d["prev"] = self.src[idx], self.tgt[idx], self.prev[idx]
        d["out"] = np.arange(n, dtype=np.int64) * crop_len
        d["nx"], d["len"] = nx, crop_len
        d["crop"] = (rng.uniform(size=n) * np.maximum(full - crop_len, 0) + 0.5).astype(np.int32)
        d["res"] = self.res[tb]
        d["cond"] = self.cond[tb]
        return d


def _upload(desc):
    import torch
    return torch.from_numpy(np.frombuffer(desc.tobytes(), dtype=np.uint8).copy()).cuda()


def train(net, cfg, data, steps, batch=32, crop_len=1024, lr=1e-3, lr_end=1e-5, margin=None,
          seed=0, noise=None, log_every=0):
    """Adam on the masked MSE of the normalised increments; cosine learning
    rate from lr to lr_end. The loss mask leaves out points closer than the
    network's receptive radius to a crop edge. ``noise`` (4 standard
    deviations of rho, u_x, theta_T, E_R) perturbs the source states, so that
    the network learns to undo errors of its own earlier windows. Returns the
    loss history."""
    import ctypes
    import torch
    lib = rpk.load_library()
    rng = np.random.default_rng(seed)
    if margin is None:
        margin = min(4 * 2 * 2 * net.nblocks, crop_len // 4)  # 2 convs x radius 2 per block, x4 fine points
    x = torch.zeros((batch, crop_len, CIN), device="cuda")
    t = torch.zeros((batch, crop_len, COUT), device="cuda")
    m = torch.zeros((batch, crop_len), device="cuda")
    nz = (ctypes.c_float * 4)(*[float(v) for v in noise]) if noise is not None else None
    hist = []
    for it in range(steps):
        idx = rng.integers(0, len(data), size=batch)
        desc = _upload(data.descriptors(idx, crop_len, cfg.pad, rng))
        rpk._check(lib.rpk_sur_pack(ctypes.byref(cfg), rpk._dev_f32(data.store), ctypes.c_void_p(desc.data_ptr()),
                                    batch, crop_len, margin, nz, seed * 1000003 + it,
                                    rpk._dev_f32(x), rpk._dev_f32(t), rpk._dev_f32(m), None))
        loss = net.loss_grad(x, t, m)
        a = lr_end + 0.5 * (lr - lr_end) * (1 + math.cos(math.pi * it / max(1, steps)))
        net.adam(a)
        hist.append(loss)
        if log_every and it % log_every == 0:
            print("step %d loss %.4e lr %.2e" % (it, loss, a), flush=True)
    return hist


def initial_blocks(tubes, fields, stream=None):
    """Moment blocks of the tubes' initial state (the LBM's moments of its
    initialised populations), as a CUDA float32 tensor."""
    bt = rpk.Batch(tubes, precision="f32", save_every=1 << 30, stream=stream)
    bt.init_fields(fields["rho"], fields["u"], fields["T"], fields["R"])
    out = bt.moments_device()
    bt.close()
    return out
