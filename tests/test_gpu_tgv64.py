"""Reduced-storage precision on the Taylor-Green vortex at Ma 0.3 (the 512^3,
Re 1600 workload copied to 64^3), against the FP64 oracle point by point.

The oracle's fields are stored in tests/golden/tgv64_*_oracle.npz by
tests/golden/make_tgv64_oracle.py (which calls only the oracle): every fourth
z plane of both sublattices after 1000 steps, as float32 deviations from the
rest state. Two copies of the 512^3 run:
  re200_paper         the 512^3 run's lattice viscosity (Re 200 on 64^3: the
                      same tau = 0.060, tau1 = 0.075 and per-step rounding of
                      the stored populations) in the paper's theta_R solver;
                      the conservative form breaks down at these relaxation
                      times in the method itself (the oracle's state turns
                      non-finite near step 850)
  re100_conservative  twice the viscosity in the default conservative form
Each storage (FP64, FP32, FP16 and BF16 deviations h = g/w - 1) runs with the
oracle's parameters and FTCS sub-step count. Errors are max|gpu - oracle| on
two scales: the full field (max|oracle|; c_s for u) and the deviation
(max|oracle - rest state|: rho = 1, u = 0, theta0, delta theta0 / 2). The
relative change of the FP64 totals M and E over the run is compared with the
oracle's own change (the paper's solver does not conserve E to round-off).
Bounds are about 3x the errors measured on GB300.
"""
import os

import numpy as np
import pytest

import paper_2201_05280_gb300 as rpk

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
T0 = 0.2948964908710633
CS = float(np.sqrt(1.4 * T0))
KEYS = ("rho", "u", "T", "Erot")
STORED = {"rho": "drho", "u": "u", "T": "dT", "Erot": "dE"}
CASES = {"re200_paper": "tgv64_re200_paper_oracle.npz",
         "re100_conservative": "tgv64_re100_conservative_oracle.npz"}

# Bounds, about 3x the errors measured on GB300: (full scale, deviation scale)
# for rho, u, theta_T, E_R, and |change of M|, |change of E| over the run minus
# the oracle's own change. FP64: the stored oracle values are float32 (2^-24
# of each deviation), and the non-FMA FP64 oracle moves its own energy total
# by 3e-12 over these 1000 steps.
BOUNDS = {
    "re200_paper": {
        "f64": ((1e-6,) * 4, (1e-6,) * 4, (1e-11, 1e-11)),
        "f32": ((1e-5, 8e-5, 3e-6, 1e-5), (1.6e-3, 1e-3, 8e-4, 1.6e-3), (4e-6, 1e-4)),
        "f16dev": ((1e-4, 8e-4, 2.5e-5, 8e-5), (1.5e-2, 1e-2, 7e-3, 1.4e-2), (4e-6, 1e-4)),
        "bf16dev": ((7e-4, 8.5e-3, 2e-4, 6.5e-4), (0.12, 0.11, 0.06, 0.11), (2e-5, 1e-4)),
    },
    "re100_conservative": {
        "f64": ((1e-6,) * 4, (1e-6,) * 4, (1e-11, 1e-11)),
        "f32": ((6e-6, 1.6e-5, 5e-6, 8e-6), (1.1e-3, 3e-4, 4.5e-4, 1.05e-3), (5e-6, 8e-6)),
        "f16dev": ((5e-5, 8e-5, 3e-5, 4e-5), (8.5e-3, 1.6e-3, 2.6e-3, 5.2e-3), (3.5e-6, 6e-6)),
        "bf16dev": ((3.6e-4, 7.6e-4, 2.4e-4, 3.5e-4), (6.5e-2, 1.5e-2, 2.1e-2, 4.5e-2), (2.2e-6, 3.4e-5)),
    },
}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    from paper_2201_05280_gb300 import build as B
    B.build()
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


def _load(case):
    z = np.load(os.path.join(HERE, "golden", CASES[case]))
    n, zs = int(z["n"]), int(z["zstride"])
    step = int(z["steps"][-1])
    ref = {k: z["%s_%d" % (STORED[k], step)].astype(np.float64) for k in KEYS}
    relax = {k: float(z["param_" + k]) for k in ("delta", "tau", "tau1", "b", "k_r")}
    relax["nsub"] = int(z["param_nsub"])
    mode = "paper" if int(z["param_rot_mode"]) == 1 else "conservative"
    return n, zs, step, ref, relax, mode, float(z["param_u0"]), z["diag0"], z["diag_%d" % step]


def _sample(a, n, zs):
    a = np.asarray(a).reshape(a.shape[:-1] + (2, n, n, n))
    return a[..., ::zs, :, :]


@pytest.mark.parametrize("case", ["re200_paper", "re100_conservative"])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16dev", "bf16dev"])
def test_taylor_green_64_storage_against_oracle(case, prec):
    import rpk_inputs as I
    n, zs, step, ref, relax, mode, u0, dg0, dg1 = _load(case)
    f = I.taylor_green(n, T0, u0)
    lat = rpk.Lattice(n, n, n, precision=prec).set_relax(**relax)
    lat.set_rot_mode(mode)
    lat.init_fields(f["rho"], f["u"], f["T"], f["R"])
    d0 = lat.diagnostics()
    lat.step(step)
    d1 = lat.diagnostics()
    got = lat.read_moments()
    lat.close()
    base = {"rho": 1.0, "u": 0.0, "T": T0, "Erot": 0.5 * relax["delta"] * T0}
    full, dev = {}, {}
    for k in KEYS:
        g = _sample(got[k], n, zs) - base[k]   # deviations, as stored
        r = ref[k]
        assert g.shape == r.shape, (k, g.shape, r.shape)
        err = np.abs(g - r).max()
        scale = max(np.abs(r).max(), CS) if k == "u" else np.abs(r + base[k]).max()
        full[k] = float(err / scale)
        dev[k] = float(err / np.abs(r).max())
    # change of the totals over the run, against the oracle's own change
    ch_or = ((dg1[0] - dg0[0]) / dg0[0], (dg1[4] - dg0[4]) / dg0[4])
    ch = ((d1["M"] - d0["M"]) / d0["M"], (d1["E"] - d0["E"]) / d0["E"])
    drift = (abs(ch[0] - ch_or[0]), abs(ch[1] - ch_or[1]))
    print("TGV64 %s %s step %d: full %s dev %s change of M, E %.3e %.3e (oracle %.3e %.3e, difference "
          "%.2e %.2e)" % (case, prec, step, {k: "%.2e" % v for k, v in full.items()},
                          {k: "%.2e" % v for k, v in dev.items()}, ch[0], ch[1], ch_or[0], ch_or[1],
                          drift[0], drift[1]))
    if prec == "f64":
        # the oracle's own totals agree with the GPU's FP64 sums
        assert abs(d0["M"] - dg0[0]) <= 1e-12 * dg0[0]
        assert abs(d1["E"] - dg1[4]) <= 1e-11 * dg1[4]
    fb, db, cb = BOUNDS[case][prec]
    for k, b in zip(KEYS, fb):
        assert full[k] <= b, ("full", k, full[k], b)
    for k, b in zip(KEYS, db):
        assert dev[k] <= b, ("deviation", k, dev[k], b)
    assert drift[0] <= cb[0] and drift[1] <= cb[1], drift
    assert d1["status"] == 0
