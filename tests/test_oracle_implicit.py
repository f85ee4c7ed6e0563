"""Pins of the oracle's backward-Euler variant of the rotational diffusion
(quasi-1-D tubes): the line solve against a dense solve of the same linear
system, its closed-form steady profile, and conservation of a full step."""
import numpy as np
import pytest

import oracle as O
from oracle import params as PM
import rpk_inputs as I

T0 = 0.2948964908710633


def _line(n, seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.2, 1.5, n)
    kap = rng.uniform(0.01, 3.0, n)
    Er = rng.uniform(0.05, 0.4, n)
    return rho, kap, Er


@pytest.mark.parametrize("n", [1, 2, 7, 64])
def test_be_line_is_the_implicit_step(n):
    delta, dt = 2.0, 1.0
    rho, kap, Er = _line(n, n)
    thl, kl, thr, kr = 0.31, 0.7, 0.22, 1.3
    got = O.diffuse_be_line(delta, dt, rho, kap, Er, thl, kl, thr, kr)
    # assemble (delta rho/2) th - dt [K+ (th+ - th) - K- (th - th-)] = Er densely
    kfull = np.concatenate([[kl], kap, [kr]])
    M = np.zeros((n, n))
    rhs = Er.copy()
    for p in range(n):
        km = 0.5 * (kfull[p + 1] + kfull[p])
        kp = 0.5 * (kfull[p + 1] + kfull[p + 2])
        M[p, p] = 0.5 * delta * rho[p] + dt * (km + kp)
        if p > 0:
            M[p, p - 1] = -dt * km
        else:
            rhs[p] += dt * km * thl
        if p < n - 1:
            M[p, p + 1] = -dt * kp
        else:
            rhs[p] += dt * kp * thr
    th = np.linalg.solve(M, rhs)
    np.testing.assert_allclose(got, 0.5 * delta * rho * th, rtol=1e-12)


def test_be_line_steady_profile_and_rest_state():
    # a huge step with uniform kappa reaches the steady profile: theta linear
    # between the two reservoir values across the n + 1 faces
    n, delta = 9, 2.0
    rho = np.full(n, 0.8)
    kap = np.ones(n)
    got = O.diffuse_be_line(delta, 1e12, rho, kap, np.full(n, 0.3), 0.4, 1.0, 0.1, 1.0)
    th = 2 * got / (delta * rho)
    np.testing.assert_allclose(th, 0.4 + (np.arange(n) + 1) * (0.1 - 0.4) / (n + 1), rtol=1e-9)
    # a uniform theta equal to both reservoirs is unchanged
    rho, kap, _ = _line(n, 3)
    Er = 0.5 * delta * rho * 0.27
    np.testing.assert_allclose(O.diffuse_be_line(delta, 5.0, rho, kap, Er, 0.27, 0.5, 0.27, 2.0), Er,
                               rtol=1e-14)


def _tube(nx, nu, diff):
    d, tau, tau1, b, kr = PM.relax_from_gas(1.4, *PM.gas_from_nondim(1.4, nu, 0.6, 0.71), 0.0)
    P = O.make_params(d, tau, tau1, b, kr, 1.0, 1, 1, diff)
    f = I.uniform(nx, 1, 1, T0)
    x = I.positions(nx, 1, 1)[0]
    bump = np.exp(-((x - nx / 2) / 6.0) ** 2)
    f["rho"] = f["rho"] * (1 + 0.05 * bump)
    f["T"] = f["T"] * (1 + 0.05 * bump)
    f["R"] = f["R"] * (1 + 0.1 * bump)
    res = np.array([1, 0, 0, 0, T0, T0] * 2, float)
    return O.State(P, nx, 1, 1, reservoirs=res).init_fields(f["rho"], f["u"], f["T"], f["R"])


def test_implicit_step_conserves_mass_momentum_energy():
    # nu = 1 gives a rotational diffusion number above the explicit limit; the
    # tube is long enough that nothing reaches the reservoirs in 20 steps
    # (populations move at most 2 cells per step)
    S = _tube(400, 1.0, 1)
    d0 = S.diag()
    S.step(20)
    d1 = S.diag()
    assert abs(d1["M"] - d0["M"]) <= 1e-12 * d0["M"]
    assert abs(d1["E"] - d0["E"]) <= 1e-12 * d0["E"]
    assert np.abs(d1["J"]).max() <= 1e-12
    F = S.fields()
    assert np.all(F["R"] > 0) and np.all(np.isfinite(F["R"]))


def test_implicit_step_close_to_explicit_for_small_diffusion_number():
    # with nu small the diffusion number is small and one implicit step differs
    # from the explicit one by O(dt^2) terms: E_R agrees to 1e-4 of its size
    # and the density, which sees E_R only through the exchange, to 1e-5
    nx = 64
    A, B = _tube(nx, 0.02, 0), _tube(nx, 0.02, 1)
    A.step(10)
    B.step(10)
    fa, fb = A.fields(), B.fields()
    assert np.abs(fa["R"] - fb["R"]).max() <= 1e-4 * np.abs(fa["R"]).max()
    assert np.abs(fa["rho"] - fb["rho"]).max() <= 1e-5


def test_implicit_variant_rejects_non_tube_grids():
    d, tau, tau1, b, kr = PM.relax_from_gas(1.4, *PM.gas_from_nondim(1.4, 0.1, 0.6, 0.71), 0.0)
    P = O.make_params(d, tau, tau1, b, kr, 1.0, 1, 0, 1)
    f = I.uniform(8, 2, 1, T0)
    S = O.State(P, 8, 2, 1).init_fields(f["rho"], f["u"], f["T"], f["R"])
    with pytest.raises(ValueError):
        S.step(1)
