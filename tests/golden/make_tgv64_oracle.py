"""Writes tgv64_oracle.npz: the FP64 oracle's moment fields of the 3-D
Taylor-Green vortex at Ma 0.3, Re 1600 (diatomic gas, eta_B/eta = 0.6,
Pr = 0.71, b = 0) on a 64^3 box of each BCC sublattice after 1000 steps.

The reduced-storage test (tests/test_gpu_tgv64.py) compares the GPU path's
FP32, FP16-deviation and BF16-deviation storage runs of the same setup with
these fields point by point. The single-threaded oracle needs about twenty
minutes for it, so its result is stored once. This script calls only
``oracle/`` and the input generator ``rpk_inputs``; nothing here comes from
the CUDA library.

Stored (float32 deviations, so that rounding the FP64 values costs at most
2^-24 of each deviation's own scale): rho - 1, u (3 x npts),
theta_T - theta0, E_R - delta theta0 / 2, at step 0 and at each step of
STEPS; the oracle's FP64 totals M, J, E at the same steps; the parameters.

    python tests/golden/make_tgv64_oracle.py [--n 64] [--steps 1000]
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

MA, RE, LAM, PR, GAMMA = 0.3, 1600.0, 0.6, 0.71, 1.4


def setup(n):
    """Fields and oracle parameters of the n^3 Taylor-Green vortex at Ma 0.3,
    Re 1600: u0 = Ma c_s, L = n/(2 pi), nu = u0 L / Re."""
    t0 = PM.THETA0
    u0 = MA * np.sqrt(GAMMA * t0)
    nu = u0 * (n / (2.0 * np.pi)) / RE
    eta, etaB, kap = PM.gas_from_nondim(GAMMA, nu, LAM, PR)
    d, tau, tau1, b, kr = PM.relax_from_gas(GAMMA, eta, etaB, kap, 0.0)
    f = I.taylor_green(n, t0, u0)
    thmax = float(np.max((3 * f["T"] + d * f["R"]) / (3 + d)))
    nsub = PM.nsub_for(d, tau, tau1, kr, thmax, 3)
    P = O.make_params(d, tau, tau1, b, kr, 1.0, nsub, 0)
    return f, P, dict(delta=d, tau=tau, tau1=tau1, b=b, k_r=kr, nsub=nsub, nu=nu, u0=u0)


def deviations(fl, delta):
    t0 = PM.THETA0
    return {"drho": (fl["rho"] - 1.0).astype(np.float32),
            "u": fl["u"].astype(np.float32),
            "dT": (fl["T"] - t0).astype(np.float32),
            "dE": (fl["Erot"] - 0.5 * delta * t0).astype(np.float32)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--steps", default="1000", help="comma-separated steps to store")
    ap.add_argument("--out", default=os.path.join(HERE, "tgv64_oracle.npz"))
    a = ap.parse_args()
    steps = sorted(int(s) for s in a.steps.split(","))
    O.build()
    f, P, prm = setup(a.n)
    S = O.State(P, a.n, a.n, a.n).init_fields(f["rho"], f["u"], f["T"], f["R"])
    out = {"n": np.int64(a.n), "steps": np.array(steps, dtype=np.int64)}
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
        dv = deviations(S.fields(), prm["delta"])
        for k, v in dv.items():
            out["%s_%d" % (k, target)] = v
        dg = S.diag()
        out["diag_%d" % target] = np.array([dg["M"], *dg["J"], dg["E"]])
    np.savez_compressed(a.out, **out)
    print("wrote", a.out, os.path.getsize(a.out), "bytes")


if __name__ == "__main__":
    main()
