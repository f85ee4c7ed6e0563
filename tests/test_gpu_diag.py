"""FP32-arithmetic diagnostics (row a9 for FP32 and 16-bit storage) against the
FP64 oracle's diagnostics of the same run.

For FP32 storage the per-point sums come from the FP32 moments (deviation
form) and are accumulated across points in FP64; H1 uses FP32 logarithms. The
state itself differs from the oracle's by FP32 rounding (~1e-7 relative after
a few steps of a smooth flow), so M, J and E agree to ~1e-7 of M and E, H1 to
~1e-6 and min g to ~1e-6 of its own size. nx even runs the two-points-per-thread
kernel, nx odd the one-point kernel, in both rotational forms (the paper's
solver holds theta_R, whose energy density delta rho theta_R / 2 enters E);
all are held to the same bars, and the 16-bit storages (whose states differ
from the oracle's by their rounding) to looser ones.
"""
import numpy as np
import pytest

import oracle as O
import paper_2201_05280_gb300 as rpk
import rpk_inputs as I

pytestmark = pytest.mark.gpu

T0 = 0.2948964908710633
RELAX = dict(delta=2.0, tau=0.6, tau1=0.8, b=0.3, k_r=0.9, nsub=2)
# (M, J, E), H1, min g; measured on GB300: FP32 7.5e-10, 1.3e-7, 1.3e-7;
# FP16 1.7e-7, 1.6e-6, 2.0e-5; BF16 1.5e-6, 1.3e-5, 1.9e-4
BARS = {"f32": (1e-8, 1e-6, 1e-6), "f16dev": (1e-6, 1e-5, 1e-4), "bf16dev": (1e-5, 1e-4, 1e-3)}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    from paper_2201_05280_gb300 import build as B
    B.build()
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("mode", ["conservative", "paper"])
@pytest.mark.parametrize("prec", ["f32", "f16dev", "bf16dev"])
@pytest.mark.parametrize("nx", [40, 41])
def test_fp32_diagnostics_against_oracle(prec, nx, mode):
    ny, nz, nsteps = 6, 4, 5
    f = I.random_smooth(nx, ny, nz, T0, seed=19)
    lat = rpk.Lattice(nx, ny, nz, precision=prec).set_relax(**RELAX)
    lat.set_rot_mode(mode)
    lat.init_fields(f["rho"], f["u"], f["T"], f["R"]).step(nsteps)
    d = lat.diagnostics()
    lat.close()
    P = O.make_params(RELAX["delta"], RELAX["tau"], RELAX["tau1"], RELAX["b"], RELAX["k_r"], 1.0,
                      RELAX["nsub"], 0, rot_mode=1 if mode == "paper" else 0)
    ref = O.State(P, nx, ny, nz).init_fields(f["rho"], f["u"], f["T"], f["R"]).step(nsteps).diag()
    cons, h1, gmin = BARS[prec]
    errs = {"M": abs(d["M"] - ref["M"]) / ref["M"],
            "J": float(np.abs(np.asarray(d["J"]) - ref["J"]).max() / ref["M"]),
            "E": abs(d["E"] - ref["E"]) / ref["E"],
            "H1": abs(d["H1"] - ref["H1"]) / abs(ref["H1"]),
            "min_g": abs(d["min_g"] - ref["min_g"]) / abs(ref["min_g"])}
    print("diagnostics %s %s nx %d: %s" % (mode, prec, nx, {k: "%.2e" % v for k, v in errs.items()}))
    assert d["status"] == 0
    assert errs["M"] <= cons and errs["J"] <= cons and errs["E"] <= cons, errs
    assert errs["H1"] <= h1, errs
    assert errs["min_g"] <= gmin, errs
