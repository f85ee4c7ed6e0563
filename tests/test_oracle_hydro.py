"""Hydrodynamic-limit pins of the oracle: decaying shear, acoustic and thermal
waves on a quasi-1-D periodic box reproduce the closed-form transport of the
model (Sec. 4, eq. viscosities and the conductivity paragraph) and the specific
heat ratio gamma = (5 + delta)/(3 + delta), within 1%.

Linearised Navier-Stokes-Fourier rates (standard results):
  shear wave      nu k^2,                      nu   = eta/rho
  thermal wave    D_T k^2,                     D_T  = kappa/(rho c_p), c_p = (5+delta)/2
  acoustic wave   omega = c_s k, c_s^2 = gamma theta0,
                  Gamma = k^2/2 [4/3 nu + eta_b/rho + (gamma - 1) D_T]
The settings keep k nu/c_s < 1e-2 and omega tau1 <= 0.05 so that Burnett and
relaxation-dispersion corrections stay well below the 1% tolerance.
"""
import numpy as np
import pytest
from scipy.optimize import curve_fit

import oracle as O
import rpk_inputs as I
from oracle import params as PM

T0 = O.THETA0
NX = 128


def _params(gamma, nu, lam, Pr, b=0.0, nx=NX):
    eta, etaB, kap = PM.gas_from_nondim(gamma, nu, lam, Pr)
    d, tau, tau1, b, kr = PM.relax_from_gas(gamma, eta, etaB, kap, b)
    P = O.make_params(d, tau, tau1, b, kr, 1.0, PM.nsub_for(d, tau, tau1, kr, T0, 1), 0)
    return P, PM.transport(d, tau, tau1, b, kr)


def _record(S, probe, every, n):
    ts, vals = [S.t], [probe(S.fields())]
    for _ in range(n // every):
        S.step(every)
        ts.append(S.t)
        vals.append(probe(S.fields()))
    return np.array(ts, float), np.array(vals)


@pytest.mark.parametrize("lam,Pr,b", [(0.6, 0.71, 0.0), (2.0, 1.4, 0.3)])
def test_shear_wave_viscosity(lam, Pr, b):
    P, tr = _params(1.4, 0.05, lam, Pr, b)
    f, k = I.shear_wave(NX, 1, 1, T0, amp=1e-4)
    S = O.State(P, NX, 1, 1).init_fields(f["rho"], f["u"], f["T"], f["R"])
    X = I.positions(NX, 1, 1)[0]
    ts, a = _record(S, lambda F: 2 * np.mean(F["u"][1] * np.sin(k * X)), 100, 2000)
    rate = -np.polyfit(ts, np.log(a), 1)[0]
    assert abs(rate / (tr["eta"] * k * k) - 1) < 0.01


def _acoustic(gamma, nu, lam, Pr, b=0.0, nsteps=2400):
    P, tr = _params(gamma, nu, lam, Pr, b)
    f, k = I.acoustic_wave(NX, 1, 1, T0, tr["gamma"], amp=1e-4)
    S = O.State(P, NX, 1, 1).init_fields(f["rho"], f["u"], f["T"], f["R"])
    X = I.positions(NX, 1, 1)[0]
    ts, bb = _record(S, lambda F: 2 * np.mean(F["u"][0] * np.sin(k * X)), 10, nsteps)
    cs = np.sqrt(tr["gamma"] * T0)
    fn = lambda t, A, G, w, ph: A * np.exp(-G * t) * np.sin(w * t + ph)
    p, _ = curve_fit(fn, ts, bb, p0=[np.abs(bb).max(), 1e-4, cs * k, 0.0])
    cp = (5 + P.delta) / 2
    G_ex = 0.5 * k * k * ((4 / 3) * tr["eta"] + tr["eta_b"] + (tr["gamma"] - 1) * tr["kappa"] / cp)
    return p, k, cs, G_ex, tr


@pytest.mark.parametrize("lam,Pr,b", [(0.6, 0.71, 0.0), (2.0, 0.71, 0.0), (1.0, 2.0, 0.5)])
def test_acoustic_wave_speed_and_attenuation(lam, Pr, b):
    p, k, cs, G_ex, tr = _acoustic(1.4, 0.05, lam, Pr, b)
    assert abs(p[2] / (cs * k) - 1) < 0.01
    assert abs(p[1] / G_ex - 1) < 0.01
    gamma_meas = (p[2] / k) ** 2 / T0
    assert abs(gamma_meas / 1.4 - 1) < 0.01


@pytest.mark.parametrize("delta", [0.03, 6.09, 30.33])
def test_specific_heat_ratio_from_sound_speed(delta):
    """Sec. 6, Table 2: the measured gamma = c_s^2/theta0 follows the imposed
    effective delta, including fractional values."""
    gamma = PM.gamma_from_delta(delta)
    p, k, cs, G_ex, tr = _acoustic(gamma, 0.05, 1.0, 0.9, nsteps=1200)
    gamma_meas = (p[2] / k) ** 2 / T0
    assert abs(gamma_meas / gamma - 1) < 0.01


@pytest.mark.parametrize("lam,Pr,b", [(0.6, 0.71, 0.0), (2.0, 3.0, 0.6)])
def test_thermal_wave_conductivity(lam, Pr, b):
    """Includes the rotational conductivity kappa_R = k_r kappa_T carried by the
    FTCS diffusion of E_R (k_r = 0.97 and 0.07 for the two cases)."""
    P, tr = _params(1.4, 0.05, lam, Pr, b)
    f, k = I.thermal_wave(NX, 1, 1, T0, amp=1e-4)
    S = O.State(P, NX, 1, 1).init_fields(f["rho"], f["u"], f["T"], f["R"])
    X = I.positions(NX, 1, 1)[0]
    d = P.delta

    def probe(F):
        th = (3 * F["T"] + d * F["R"]) / (3 + d)
        return 2 * np.mean(th * np.sin(k * X))

    ts, a = _record(S, probe, 20, 2000)
    rate = -np.polyfit(ts[5:], np.log(a[5:]), 1)[0]
    cp = (5 + d) / 2
    assert abs(rate / (tr["kappa"] / cp * k * k) - 1) < 0.01
