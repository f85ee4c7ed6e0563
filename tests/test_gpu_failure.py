"""Failure detection on the GPU path, driven by host-chosen inputs only (no
device fault, trap or hang is involved).

1. Numerical breakdown: the full-strength Sod tube (rho 1/0.125, p 1/0.1,
   2000 cells, Kn 1e-3) leaves the positivity region of the third-order
   Hermite equilibrium at the shock; the FP64 oracle's state itself turns
   non-finite between steps 900 and 925. The collide kernel's status word
   must then make rpk_diagnostics and rpk_read_moments return
   RPK_ERR_NUMERIC (4), while the same run at step 400 reports no fault.
2. Invalid initial fields, on the host or already on the device, are
   refused with RPK_ERR_PARAM (2) before any step.
"""
import numpy as np
import pytest

import oracle as O
import paper_2201_05280_gb300 as rpk
import rpk_inputs as I

pytestmark = pytest.mark.gpu

T0 = 0.2948964908710633


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    from paper_2201_05280_gb300 import build as B
    B.build()
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


def _sod():
    nx = 2000
    nu = 1e-3 * rpk.sound_speed(1.4) * nx  # Kn = nu / (c_s L)
    eta, etaB, kap = rpk.gas_from_nondim(1.4, nu, 0.6, 0.71)
    r = rpk.map_gas(1.4, eta, etaB, kap, 0.0)
    relax = {k: r[k] for k in ("delta", "tau", "tau1", "b", "k_r")}
    f, res = I.shock_tube(nx, T0)
    return nx, f, res, relax


def test_numeric_breakdown_is_reported_as_err_numeric():
    nx, f, res, relax = _sod()
    lat = rpk.Lattice(nx, 1, 1, precision="f64", bc_x="reservoir").set_relax(**relax)
    lat.set_reservoirs(res)
    lat.init_fields(f["rho"], f["u"], f["T"], f["R"])
    nsub = lat.info()["nsub"]
    lat.step(400)
    d = lat.diagnostics()  # raises on a flagged state
    assert d["status"] == 0 and np.isfinite(d["E"])
    lat.step(600)
    with pytest.raises(rpk.RpkError) as e:
        lat.diagnostics()
    assert e.value.code == 4
    d = lat.diagnostics(check=False)
    assert d["status"] != 0
    with pytest.raises(rpk.RpkError) as e:
        lat.read_moments()
    assert e.value.code == 4
    lat.close()
    # the method itself breaks down on this input: the FP64 oracle's state is
    # no longer finite after the same 1000 steps
    P = O.make_params(relax["delta"], relax["tau"], relax["tau1"], relax["b"], relax["k_r"],
                      1.0, nsub, 1)
    S = O.State(P, nx, 1, 1, reservoirs=res).init_fields(f["rho"], f["u"], f["T"], f["R"])
    S.step(1000)
    assert not np.all(np.isfinite(S.fields()["rho"]))


@pytest.mark.parametrize("where", ["host", "device"])
@pytest.mark.parametrize("bad", ["rho_zero", "T_negative", "R_nan", "u_inf"])
def test_invalid_initial_fields_are_refused(where, bad):
    import torch
    nx, ny, nz = 6, 5, 4
    f = I.random_smooth(nx, ny, nz, T0, seed=2)
    g = {k: np.array(v, dtype=np.float64, copy=True) for k, v in f.items()}
    if bad == "rho_zero":
        g["rho"][7] = 0.0
    elif bad == "T_negative":
        g["T"][11] = -T0
    elif bad == "R_nan":
        g["R"][3] = np.nan
    else:
        g["u"][1, 5] = np.inf
    if where == "device":
        g = {k: torch.from_numpy(np.ascontiguousarray(v).reshape(-1)).cuda() for k, v in g.items()}
    lat = rpk.Lattice(nx, ny, nz, precision="f32").set_relax(delta=2.0, tau=0.6, tau1=0.8)
    with pytest.raises(rpk.RpkError) as e:
        lat.init_fields(g["rho"], g["u"], g["T"], g["R"])
    assert e.value.code == 2
    with pytest.raises(rpk.RpkError) as e:
        lat.step(1)
    assert e.value.code == 5  # nothing was initialised
    lat.init_fields(f["rho"], f["u"], f["T"], f["R"]).step(2)
    assert lat.diagnostics()["status"] == 0
    lat.close()
