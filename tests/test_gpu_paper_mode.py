"""GPU parity of the paper-mode rotational solver (rpk_set_rot_mode(1): the
four steps of Sec. 5 on theta_R) against the oracle's paper mode, on the same
seeded inputs: FP64 relative L-inf 1e-12 per field (u on the c_s scale),
FP32 1e-5 after 500 steps of a smooth flow; periodic 3-D boxes with ragged
sizes and a shock tube with reservoirs; checkpoints keep the mode."""
import numpy as np
import pytest

import oracle as O
import paper_2201_05280_gb300 as rpk
import rpk_inputs as I

pytestmark = pytest.mark.gpu

T0 = 0.2948964908710633
CS = np.sqrt(1.4 * T0)
RELAX = dict(delta=2.0, tau=0.6, tau1=0.8, b=0.3, k_r=0.9, nsub=2)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2201_05280_gb300 import build as B
    B.build()
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


def _run(nx, ny, nz, f, relax, nsteps, precision="f64", bcx=0, res=None):
    lat = rpk.Lattice(nx, ny, nz, precision=precision, bc_x="reservoir" if bcx else "periodic")
    lat.set_relax(**relax)
    lat.set_rot_mode("paper")
    if bcx:
        lat.set_reservoirs(res)
    lat.init_fields(f["rho"], f["u"], f["T"], f["R"])
    nsub = lat.info()["nsub"]
    P = O.make_params(relax["delta"], relax["tau"], relax["tau1"], relax.get("b", 0.0),
                      relax.get("k_r", 0.0), 1.0, nsub, bcx, 0, 1)
    S = O.State(P, nx, ny, nz, reservoirs=res).init_fields(f["rho"], f["u"], f["T"], f["R"])
    lat.step(nsteps)
    S.step(nsteps)
    return lat.read_moments(), S.fields(), lat


def _errs(got, ref):
    e = {k: float(np.abs(got[k] - ref[k]).max() / np.abs(ref[k]).max()) for k in ("rho", "T", "R", "Erot")}
    e["u"] = float(np.abs(got["u"] - ref["u"]).max() / max(np.abs(ref["u"]).max(), CS))
    return e


@pytest.mark.parametrize("dims", [(5, 4, 3), (33, 2, 1), (1, 1, 1)])
def test_paper_mode_f64_periodic(dims):
    f = I.random_smooth(*dims, T0, seed=41, amp=0.02, aniso_R=0.02)
    got, ref, lat = _run(*dims, f, RELAX, 200)
    e = _errs(got, ref)
    assert max(e.values()) <= 1e-12, e
    lat.close()


def test_paper_mode_f64_shock_tube_with_reservoirs():
    f, res = I.shock_tube(96, T0, rho_r=1 / 1.5, p_r=0.5)
    relax = dict(delta=2.0, tau=0.5, tau1=0.9, b=0.0, k_r=0.8, nsub=3)
    got, ref, lat = _run(96, 1, 1, f, relax, 150, bcx=1, res=res)
    e = _errs(got, ref)
    assert max(e.values()) <= 1e-12, e
    lat.close()


def test_paper_mode_f32_smooth_500_steps():
    f = I.random_smooth(24, 6, 4, T0, seed=43, amp=0.01, aniso_R=0.01)
    got, ref, lat = _run(24, 6, 4, f, RELAX, 500, precision="f32")
    e = _errs(got, ref)
    assert max(e.values()) <= 1e-5, e
    lat.close()


def test_paper_mode_diagnostics_and_checkpoint(tmp_path):
    f = I.random_smooth(6, 5, 4, T0, seed=44)
    got, ref, lat = _run(6, 5, 4, f, RELAX, 30)
    d = lat.diagnostics()
    P = O.make_params(2.0, 0.6, 0.8, 0.3, 0.9, 1.0, 2, 0, 0, 1)
    S = O.State(P, 6, 5, 4).init_fields(f["rho"], f["u"], f["T"], f["R"])
    S.step(30)
    dref = S.diag()
    assert abs(d["M"] - dref["M"]) <= 1e-12 * dref["M"]
    assert abs(d["E"] - dref["E"]) <= 1e-12 * dref["E"]
    path = str(tmp_path / "pm.ckpt")
    lat.save(path)
    lat.step(10)
    a = lat.read_moments()
    other = rpk.Lattice(6, 5, 4, precision="f64")
    other.set_relax(**RELAX)
    with pytest.raises(rpk.RpkError):
        other.load(path)  # conservative lattice, paper-mode checkpoint
    other.set_rot_mode("paper").load(path)
    other.step(10)
    b = other.read_moments()
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])
    lat.close()
    other.close()
