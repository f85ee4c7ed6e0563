"""Pins of the host-side parameter mapping (oracle side) against the numbers the
paper prints: Table 2 (gamma vs effective delta) and Table 3 (Landau numbers),
and the relation lambda = 224/(225 Pr) stated for tau = (3/5) tau1 (Sec. 6)."""
import os

import numpy as np
import pytest

from oracle import params as PM

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _table(name):
    return np.loadtxt(os.path.join(GOLD, name), comments="#")


def test_table2_gamma_of_delta():
    for gamma, delta in _table("effective_delta_table2.txt"):
        # the table prints gamma to 2-4 significant digits
        assert abs(PM.gamma_from_delta(delta) - gamma) <= 0.0051 * gamma
        assert abs(PM.delta_from_gamma(PM.gamma_from_delta(delta)) - delta) < 1e-12


def test_table3_landau_numbers():
    """tau = (3/5) tau1, k_r = 0, gamma = 7/5: the mapping gives lambda = eta_b/eta
    = 224/(225 Pr) and La = Kn (4/3 + lambda) + Kn (gamma - 1)/Pr."""
    Kn = 1e-3
    delta = PM.delta_from_gamma(1.4)
    for Pr, La in _table("landau_table3.txt"):
        # choose b so that the model's Pr comes out with tau = 0.6 tau1, k_r = 0
        tau1 = 1.0
        tau = 0.6 * tau1
        B = 1 + tau / tau1
        b = B - B * (1 + delta / 5) / Pr
        tr = PM.transport(delta, tau, tau1, b, 0.0)
        assert abs(tr["Pr"] - Pr) < 1e-12
        lam = tr["eta_b"] / tr["eta"]
        assert abs(lam - 224 / (225 * Pr)) < 1e-12
        La_model = Kn * (4 / 3 + lam) + Kn * (tr["gamma"] - 1) / Pr
        assert abs(La_model - La) < 0.6e-7  # table rounding in the 5th digit


@pytest.mark.parametrize("gamma,nu,lam,Pr,b", [(1.4, 0.05, 0.6, 0.71, 0.0),
                                               (1.4, 1.285, 0.6, 0.71, 0.0),
                                               (1.31, 0.02, 2.0, 1.3, 0.4),
                                               (1.66, 0.1, 0.9, 0.67, -0.3)])
def test_mapping_round_trip(gamma, nu, lam, Pr, b):
    eta, etaB, kap = PM.gas_from_nondim(gamma, nu, lam, Pr)
    d, tau, tau1, b2, kr = PM.relax_from_gas(gamma, eta, etaB, kap, b)
    tr = PM.transport(d, tau, tau1, b2, kr)
    assert abs(tr["eta"] - eta) < 1e-12 * eta
    assert abs(tr["eta_b"] - etaB) < 1e-12 * etaB
    assert abs(tr["kappa"] - kap) < 1e-12 * kap
    assert abs(tr["Pr"] - Pr) < 1e-12
    assert abs(tr["gamma"] - gamma) < 1e-12


def test_bulk_ratio_below_c_delta_needs_b_above_one():
    """eta_b/eta >= c_delta = 2 delta/(3(3 + delta)) whenever b <= 1 (from
    eq. viscosities); below it no positive tau exists."""
    delta = 2.0
    assert abs(PM.c_delta(delta) - 4.0 / 15.0) < 1e-15
    with pytest.raises(ValueError):
        PM.relax_from_gas(1.4, 0.05, 0.2 * 0.05, 1.0, 0.0)
