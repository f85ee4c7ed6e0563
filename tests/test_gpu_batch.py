"""GPU parity of the batched quasi-1-D tubes (rpk_batch_*): every tube of a
batch must match the FP64 oracle run of the same nx x 1 x 1 lattice with x
reservoirs, both the final state and the snapshots taken during the run.
FP64 tolerance as in test_gpu_parity (u on the scale max(|u|, c_s)). FP32
shock tubes have deviations |h| up to about 2 (density ratios up to 8), so the
round-to-nearest of the stored h adds about 2^-24 * 2 per step and up to 1e-5
over the 80 steps here; their bound is 5e-5. Snapshots are stored as float32
and compared at 1e-6 (or the run's bound when larger)."""
import numpy as np
import pytest

import oracle as O
import paper_2201_05280_gb300 as rpk
import rpk_inputs as I
from oracle import params as PM

pytestmark = pytest.mark.gpu

T0 = 0.2948964908710633
CS = np.sqrt(1.4 * T0)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    from paper_2201_05280_gb300 import build as B
    B.build()
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


def _relax_for(spec, fields_T, fields_R):
    """Raw parameters of one tube: nu = Kn c_s L, eta_B/eta and Pr from the
    spec; the oracle's mapping, with nsub from its own FTCS rule."""
    nu = spec["kn"] * CS * spec["nx"]
    eta, etaB, kap = PM.gas_from_nondim(1.4, nu, spec["lam"], spec["pr"])
    d, tau, tau1, b, kr = PM.relax_from_gas(1.4, eta, etaB, kap, 0.0)
    thmax = max(float(np.max((3 * fields_T + d * fields_R) / (3 + d))),
                float(np.max((3 * spec["res"][[4, 10]] + d * spec["res"][[5, 11]]) / (3 + d))))
    nsub = PM.nsub_for(d, tau, tau1, kr, thmax, 1)
    return dict(delta=d, tau=tau, tau1=tau1, b=b, k_r=kr, nsub=nsub)


def _setup(ntubes, L, seed, nsteps_cap=None, ratio=(2.0, 20.0)):
    specs, f = I.tube_sweep(ntubes, T0, seed=seed, L=L, ratio=ratio)
    tubes = []
    for i, sp in enumerate(specs):
        lo, hi = 2 * sum(s["nx"] for s in specs[:i]), 2 * sum(s["nx"] for s in specs[:i + 1])
        relax = _relax_for(sp, f["T"][lo:hi], f["R"][lo:hi])
        nsteps = sp["nsteps"] if nsteps_cap is None else min(sp["nsteps"], nsteps_cap)
        tubes.append({"nx": sp["nx"], "nsteps": nsteps, "relax": relax, "res": sp["res"],
                      "lo": lo, "hi": hi})
    return tubes, f


def _oracle_tube(t, f, save_every, nruns=1, diff=0):
    r = t["relax"]
    P = O.make_params(r["delta"], r["tau"], r["tau1"], r["b"], r["k_r"], 1.0, r["nsub"], 1, diff)
    lo, hi = t["lo"], t["hi"]
    S = O.State(P, t["nx"], 1, 1, reservoirs=t["res"]).init_fields(
        f["rho"][lo:hi], f["u"][:, lo:hi], f["T"][lo:hi], f["R"][lo:hi])
    snaps = []
    for run in range(nruns):
        done = 0
        while done < t["nsteps"]:
            if run == nruns - 1:
                F = S.fields()
                snaps.append(np.stack([F["rho"], F["u"][0], F["T"], F["Erot"]]))
            k = min(save_every, t["nsteps"] - done)
            S.step(k)
            done += k
    return S.fields(), snaps


def _cmp(got, ref, tol):
    errs = {}
    for k in ("rho", "T", "R", "Erot"):
        errs[k] = float(np.abs(got[k] - ref[k]).max() / np.abs(ref[k]).max())
    errs["u"] = float(np.abs(got["u"] - ref["u"]).max() / max(np.abs(ref["u"]).max(), CS))
    assert all(v <= tol for v in errs.values()), errs
    return errs


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 5e-5)])
def test_batch_matches_oracle_per_tube(prec, tol):
    save_every = 8
    tubes, f = _setup(6, (24, 160), seed=5)
    B = rpk.Batch(tubes, precision=prec, save_every=save_every)
    B.init_fields(f["rho"], f["u"], f["T"], f["R"]).run()
    got = B.read_moments()
    snaps = B.snapshots()
    for i, t in enumerate(tubes):
        ref, ref_snaps = _oracle_tube(t, f, save_every)
        lo, hi = t["lo"], t["hi"]
        g = {k: (got[k][:, lo:hi] if k == "u" else got[k][lo:hi]) for k in got}
        _cmp(g, ref, tol)
        assert snaps[i].shape == (len(ref_snaps), 4, hi - lo)
        for a, b in zip(snaps[i], ref_snaps):
            for j in (0, 2, 3):
                assert np.abs(a[j] - b[j]).max() <= max(1e-6, tol) * np.abs(b[j]).max()
            assert np.abs(a[1] - b[1]).max() <= max(1e-6, tol) * max(np.abs(b[1]).max(), CS)
    B.close()


def test_batch_launch_configs_agree_bitwise_and_autotune():
    tubes, f = _setup(40, (16, 300), seed=9, nsteps_cap=40)
    results = []
    for threads in (128, 512):
        B = rpk.Batch(tubes, precision="f32", save_every=16)
        B.init_fields(f["rho"], f["u"], f["T"], f["R"]).set_config(threads).run()
        results.append(B.read_moments())
        B.close()
    for k in results[0]:
        np.testing.assert_array_equal(results[0][k], results[1][k])
    B = rpk.Batch(tubes, precision="f32", save_every=16)
    B.init_fields(f["rho"], f["u"], f["T"], f["R"])
    cfg = B.autotune()
    assert cfg["threads"] in (128, 256, 384, 512) and cfg["ctas_per_sm"] >= 1
    B.run()
    for k, v in B.read_moments().items():
        np.testing.assert_array_equal(v, results[0][k])
    B.close()


def test_batch_second_run_continues_the_tubes():
    save_every = 10
    tubes, f = _setup(3, (40, 90), seed=13, nsteps_cap=30)
    B = rpk.Batch(tubes, precision="f64", save_every=save_every)
    B.init_fields(f["rho"], f["u"], f["T"], f["R"]).run().run()
    got = B.read_moments()
    snaps = B.snapshots()
    for i, t in enumerate(tubes):
        ref, ref_snaps = _oracle_tube(t, f, save_every, nruns=2)
        lo, hi = t["lo"], t["hi"]
        g = {k: (got[k][:, lo:hi] if k == "u" else got[k][lo:hi]) for k in got}
        _cmp(g, ref, 1e-12)
        assert np.abs(snaps[i][-1][0] - ref_snaps[-1][0]).max() <= 1e-6
    B.close()


def test_batch_longest_tube_fits_shared_memory():
    nmax = rpk.Batch.max_nx("f32")
    assert nmax >= 4000  # the sweep's longest tubes
    tubes, f = _setup(1, (nmax, nmax), seed=3, nsteps_cap=12)
    B = rpk.Batch(tubes, precision="f32", save_every=4)
    B.init_fields(f["rho"], f["u"], f["T"], f["R"]).run()
    got = B.read_moments()
    ref, _ = _oracle_tube(tubes[0], f, 4)
    _cmp(got, ref, 1e-5)
    B.close()
    with pytest.raises(rpk.RpkError):
        rpk.Batch([dict(tubes[0], nx=nmax + 1)], precision="f32")


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 5e-5)])
def test_batch_implicit_diffusion_matches_oracle(prec, tol):
    """The backward-Euler variant (cyclic reduction on the GPU, Thomas in the
    oracle) on tubes with large and small diffusion numbers, including one
    tube of odd length and one of a single cell pair."""
    save_every = 16
    tubes, f = _setup(6, (24, 300), seed=31, nsteps_cap=60)
    B = rpk.Batch(tubes, precision=prec, save_every=save_every)
    B.set_diffusion("implicit")
    B.init_fields(f["rho"], f["u"], f["T"], f["R"]).run()
    got = B.read_moments()
    for i, t in enumerate(tubes):
        ref, _ = _oracle_tube(t, f, save_every, diff=1)
        lo, hi = t["lo"], t["hi"]
        g = {k: (got[k][:, lo:hi] if k == "u" else got[k][lo:hi]) for k in got}
        _cmp(g, ref, tol)
    B.close()


def test_batch_implicit_tiny_and_odd_tubes():
    # weak pressure ratios: a strong shock on a few cells breaks the Hermite-3
    # populations' positivity in the oracle too
    tubes, f = _setup(5, (2, 9), seed=38, ratio=(2.0, 2.5))
    for t in tubes:
        t["nsteps"] = 20
    assert sorted({t["nx"] % 2 for t in tubes}) == [0, 1]
    B = rpk.Batch(tubes, precision="f64", save_every=8)
    B.set_diffusion("implicit")
    B.init_fields(f["rho"], f["u"], f["T"], f["R"]).run()
    got = B.read_moments()
    for t in tubes:
        ref, _ = _oracle_tube(t, f, 8, diff=1)
        lo, hi = t["lo"], t["hi"]
        _cmp({k: (got[k][:, lo:hi] if k == "u" else got[k][lo:hi]) for k in got}, ref, 1e-12)
    B.close()
