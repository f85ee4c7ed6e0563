"""CPU checks of the C interface: the library builds and loads, exports every
entry point that include/rpk.h declares, and its host-only functions (the
parameter mapping of Sec. 4 and the FTCS sub-step rule) agree with the oracle's
independent versions. No compute call is made here (no GPU)."""
import os
import re

import numpy as np
import pytest

import oracle.params as PM
import paper_2201_05280_gb300 as rpk
from paper_2201_05280_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return rpk.load_library()


def _declared():
    text = open(os.path.join(ROOT, "include", "rpk.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rpk_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n


def test_only_the_c_interface_is_exported(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", rpk.library_path()],
                         capture_output=True, text=True).stdout
    text_syms = [l.split()[-1] for l in out.splitlines() if " T " in l]
    assert text_syms and all(s.startswith("rpk_") for s in text_syms)
    assert sorted(text_syms) == _declared()


def test_theta0_and_abi(lib):
    assert rpk.theta0() == 0.2948964908710633
    assert lib.rpk_abi_version() == 1


@pytest.mark.parametrize("gamma,nu,lam,Pr,b", [(1.4, 0.05, 0.6, 0.71, 0.0),
                                               (1.4, 1.285, 0.6, 0.71, 0.0),
                                               (1.31, 0.02, 2.0, 1.3, 0.4),
                                               (1.66, 0.1, 0.9, 0.67, -0.3)])
def test_map_gas_matches_oracle_mapping(lib, gamma, nu, lam, Pr, b):
    eta, etaB, kap = rpk.gas_from_nondim(gamma, nu, lam, Pr)
    assert np.allclose((eta, etaB, kap), PM.gas_from_nondim(gamma, nu, lam, Pr), rtol=1e-15)
    got = rpk.map_gas(gamma, eta, etaB, kap, b)
    ref = PM.relax_from_gas(gamma, eta, etaB, kap, b)
    for k, v in zip(("delta", "tau", "tau1", "b", "k_r"), ref):
        assert abs(got[k] - v) <= 1e-13 * max(1.0, abs(v)), (k, got[k], v)
    assert got["dt"] == 1.0 and got["nsub"] == 0


def test_map_gas_rejects_unreachable_bulk_ratio(lib):
    with pytest.raises(rpk.RpkError) as e:
        rpk.map_gas(1.4, 0.05, 0.2 * 0.05, 0.3, 0.0)
    assert e.value.code == 2 and "b > 1" in str(e.value)
    with pytest.raises(rpk.RpkError):
        rpk.map_gas(1.7, 0.05, 0.03, 0.3, 0.0)


@pytest.mark.parametrize("theta_max,ndim", [(0.2949, 1), (0.35, 3), (0.29, 2)])
def test_auto_nsub_matches_oracle_rule(lib, theta_max, ndim):
    for tau, tau1, kr in [(7.84, 9.80, 0.97), (0.3, 0.38, 0.97), (1.0, 2.0, 0.0), (2.0, 0.5, 4.0)]:
        r = {"delta": 2.0, "tau": tau, "tau1": tau1, "b": 0.0, "k_r": kr, "dt": 1.0, "nsub": 0}
        assert rpk.auto_nsub(r, theta_max, ndim) == PM.nsub_for(2.0, tau, tau1, kr, theta_max, ndim)


def test_gas_from_nondim_in_the_library(lib):
    """The Sec. 4 relations the binding no longer computes itself: the
    library's (eta, eta_B, kappa) against the oracle's mapping, a hand value
    for air (delta = 2: c_p = 7/2, so kappa = 7 eta / (2 Pr)) and the errors."""
    eta, etaB, kap = rpk.gas_from_nondim(1.4, 0.02, 0.6, 0.71)
    assert (eta, etaB) == (0.02, 0.6 * 0.02)
    assert abs(kap - 3.5 * 0.02 / 0.71) <= 1e-16
    for bad in ((1.0, 0.02, 0.6, 0.71), (1.4, 0.0, 0.6, 0.71), (1.4, 0.02, 0.6, -1.0),
                (1.4, float("nan"), 0.6, 0.71)):
        with pytest.raises(rpk.RpkError) as e:
            rpk.gas_from_nondim(*bad)
        assert e.value.code == 2


def test_sound_speed_and_nsub_of_fields(lib):
    t0 = PM.THETA0
    assert abs(rpk.sound_speed(1.4) - np.sqrt(1.4 * t0)) <= 1e-16
    assert np.isnan(rpk.sound_speed(1.8))
    rng = np.random.default_rng(3)
    T = t0 * (1 + 0.3 * rng.random(50))
    R = t0 * (1 + 0.3 * rng.random(50))
    res = [1.0, 0, 0, 0, 2.0 * t0, 1.5 * t0, 0.5, 0, 0, 0, t0, t0]
    r = {"delta": 2.0, "tau": 0.9, "tau1": 1.1, "b": 0.0, "k_r": 3.0, "dt": 1.0, "nsub": 0}
    theta = (3 * T + 2.0 * R) / 5.0
    assert rpk.auto_nsub_fields(r, T, R, None, 3) == PM.nsub_for(2.0, 0.9, 1.1, 3.0, theta.max(), 3)
    # the hotter reservoir decides
    assert rpk.auto_nsub_fields(r, T, R, res, 1) == PM.nsub_for(2.0, 0.9, 1.1, 3.0, 1.8 * t0, 1)


def test_tube_reservoirs_in_the_library(lib):
    t0 = PM.THETA0
    tube = {"nx": 10, "nsteps": 5, "relax": {"delta": 2.0, "tau": 1.0, "tau1": 1.0},
            "res": [1.0, 0.1, 0, 0, t0, 1.2 * t0, 0.4, 0.0, 0, 0, 0.8 * t0, 0.9 * t0]}
    got = rpk.tube_reservoirs(tube)
    # E_R = delta rho theta_R / 2
    ref = np.array([[1.0, 0.1, t0, 1.2 * t0], [0.4, 0.0, 0.8 * t0, 0.4 * 0.9 * t0]], np.float32)
    assert np.array_equal(got, ref)


def test_gpu_calls_fail_loudly_without_a_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(rpk.RpkError) as e:
        rpk.Lattice(4, 4, 4)
    assert e.value.code == 3


def test_missing_library_raises(tmp_path):
    import importlib
    mod = importlib.import_module("paper_2201_05280_gb300")
    saved = mod._lib
    try:
        mod._lib = None
        with pytest.raises(ImportError):
            mod.load_library(str(tmp_path / "nope.so"))
    finally:
        mod._lib = saved
