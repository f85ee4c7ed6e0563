"""Writes tgv64_<case>_oracle.npz: the FP64 oracle's moment fields of the
3-D Taylor-Green vortex at Ma 0.3 (diatomic gas, eta_B/eta = 0.6, Pr = 0.71,
b = 0) on a 64^3 box of each BCC sublattice, after 1000 steps.

The 512^3 Taylor-Green vortex at Ma 0.3, Re 1600 copied to 64^3 with the same
lattice viscosity (nu = u0 L / Re with L eight times smaller, i.e. Re 200 on
64^3), hence the same relaxation times (tau = 0.060, tau1 = 0.075) and the
same per-step rounding regime of the stored populations. With these
relaxation times the conservative form of the rotational energy breaks down
(a mode grows from round-off by e every ~20 steps; the oracle's state turns
non-finite near step 850), while the paper's own theta_R solver stays stable.
Two cases:
  --re 200 --mode paper          the 512^3 relaxation times, paper's solver
  --re 100 --mode conservative   twice the viscosity, the default solver

The reduced-storage test (tests/test_gpu_tgv64.py) compares the GPU path's
FP32, FP16-deviation and BF16-deviation storage runs of the same setups with
these fields point by point. The single-threaded oracle needs about half an
hour for 1000 steps, so its results are stored once. This script calls only
``oracle/`` and the input generator ``rpk_inputs``; nothing here comes from
the CUDA library.

Stored, on every fourth z plane (z = 0, 4, ..., 60) of both sublattices, as
float32 deviations (rounding the FP64 values costs at most 2^-24 of each
deviation's own scale): rho - 1, u (3 components), theta_T - theta0,
E_R - delta theta0 / 2 at each step of STEPS; the oracle's FP64 totals M, J, E
at step 0 and at those steps; the parameters.

    python tests/golden/make_tgv64_oracle.py --re 200 --mode paper
    python tests/golden/make_tgv64_oracle.py --re 100 --mode conservative
"""
import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from oracle import params as PM  # noqa: E402
import rpk_inputs as I  # noqa: E402

MA, LAM, PR, GAMMA = 0.3, 0.6, 0.71, 1.4
ZSTRIDE = 4  # stored z planes: 0, 4, 8, ...


def setup(n, re, rot_mode):
    """Fields and oracle parameters of the n^3 Taylor-Green vortex at Ma 0.3
    and Reynolds number re: u0 = Ma c_s, L = n/(2 pi), nu = u0 L / re;
    rot_mode 0 = conservative rotational energy, 1 = the paper's solver."""
    t0 = PM.THETA0
    u0 = MA * np.sqrt(GAMMA * t0)
    nu = u0 * (n / (2.0 * np.pi)) / re
    eta, etaB, kap = PM.gas_from_nondim(GAMMA, nu, LAM, PR)
    d, tau, tau1, b, kr = PM.relax_from_gas(GAMMA, eta, etaB, kap, 0.0)
    f = I.taylor_green(n, t0, u0)
    thmax = float(np.max((3 * f["T"] + d * f["R"]) / (3 + d)))
    nsub = PM.nsub_for(d, tau, tau1, kr, thmax, 3)
    P = O.make_params(d, tau, tau1, b, kr, 1.0, nsub, 0, rot_mode=rot_mode)
    return f, P, dict(delta=d, tau=tau, tau1=tau1, b=b, k_r=kr, nsub=nsub, nu=nu, u0=u0,
                      rot_mode=rot_mode)


def sample(a, n):
    """Every ZSTRIDE-th z plane of a field (..., 2, n, n, n) in [s][z][y][x]."""
    a = np.asarray(a).reshape(a.shape[:-1] + (2, n, n, n))
    return np.ascontiguousarray(a[..., ::ZSTRIDE, :, :])


def deviations(fl, delta, n):
    t0 = PM.THETA0
    return {"drho": sample(fl["rho"] - 1.0, n).astype(np.float32),
            "u": sample(fl["u"], n).astype(np.float32),
            "dT": sample(fl["T"] - t0, n).astype(np.float32),
            "dE": sample(fl["Erot"] - 0.5 * delta * t0, n).astype(np.float32)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--re", type=float, default=200.0)
    ap.add_argument("--mode", choices=["paper", "conservative"], default="paper")
    ap.add_argument("--steps", default="1000", help="comma-separated steps to store")
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    out_path = a.out or os.path.join(HERE, "tgv%d_re%d_%s_oracle.npz" % (a.n, int(a.re), a.mode))
    steps = sorted(int(s) for s in a.steps.split(","))
    O.build()
    f, P, prm = setup(a.n, a.re, 1 if a.mode == "paper" else 0)
    S = O.State(P, a.n, a.n, a.n).init_fields(f["rho"], f["u"], f["T"], f["R"])
    out = {"n": np.int64(a.n), "re": np.float64(a.re), "zstride": np.int64(ZSTRIDE),
           "steps": np.array(steps, dtype=np.int64)}
    for k, v in prm.items():
        out["param_" + k] = np.float64(v)
    d0 = S.diag()
    out["diag0"] = np.array([d0["M"], *d0["J"], d0["E"]])
    t = 0
    t_start = time.time()
    for target in steps:
        while t < target:
            k = min(50, target - t)
            S.step(k)
            t += k
            fl = S.fields()
            print("step %d  max|u| %.4f  min rho %.4f  min T %.4f  (%.0f s)"
                  % (t, np.abs(fl["u"]).max(), fl["rho"].min(), fl["T"].min(),
                     time.time() - t_start), flush=True)
            if not np.all(np.isfinite(fl["rho"])):
                raise SystemExit("oracle state not finite at step %d" % t)
        dv = deviations(S.fields(), prm["delta"], a.n)
        for k, v in dv.items():
            out["%s_%d" % (k, target)] = v
        dg = S.diag()
        out["diag_%d" % target] = np.array([dg["M"], *dg["J"], dg["E"]])
    np.savez_compressed(out_path, **out)
    print("wrote", out_path, os.path.getsize(out_path), "bytes")


if __name__ == "__main__":
    main()
