"""Pins of the oracle's single-point collision against the paper's definitions:
the trapezoid transform g = f - (dt/2) Omega (Sec. 5), the zero of collision
(Sec. 4, hydrodynamics paragraph), closed-form homogeneous relaxation of the
discrete scheme, and conservation at one point (Sec. 4, eq. ConservedMomEq)."""
import numpy as np
import pytest

import oracle as O

T0 = O.THETA0
DT = 1.0


def _params(delta=2.0, tau=0.7, tau1=0.9, b=0.3, kr=0.5):
    return O.make_params(delta, tau, tau1, b, kr, DT, 1, 0)


def _fmoments(f, c):
    rho = f.sum()
    u = f @ c / rho
    P = np.einsum("i,ia,ib->ab", f, c, c)
    T = (np.trace(P) - rho * u @ u) / (3 * rho)
    sigma = P - rho * np.outer(u, u) - rho * T * np.eye(3)
    return rho, u, T, sigma


def _g_from_f(P, f, R, c):
    """Direct use of the definitions: Omega of Sec. 5 evaluated on f with the
    targets f^ES(rho, u, T I + b sigma/rho) and f^Eq(rho, u, theta I), and the
    same trapezoid shift for the rotational energy of eq. kinEqBGK."""
    rho, u, T, sigma = _fmoments(f, c)
    theta = (3 * T + P.delta * R) / (3 + P.delta)
    fES = O.target(rho, u, T * np.eye(3) + P.b * sigma / rho)
    fEq = O.target(rho, u, theta * np.eye(3))
    Omega = (fES - f) / P.tau + (fEq - f) / P.tau1
    g = f - 0.5 * DT * Omega
    ER = 0.5 * P.delta * rho * R
    Er = ER - 0.5 * DT * (0.5 * P.delta * rho) * (theta - R) / P.tau1
    return g, Er, (rho, u, T, sigma, theta)


@pytest.mark.parametrize("seed", range(4))
def test_recovery_inverts_the_trapezoid_transform(seed):
    """From (g, Er) built by the definitions, the oracle recovers the f-level
    theta_T, theta_R and sigma (the g/f moment relations of Sec. 5), and f."""
    rng = np.random.default_rng(seed)
    c, w = O.lattice()
    P = _params(tau=rng.uniform(0.3, 3), tau1=rng.uniform(0.3, 3), b=rng.uniform(-0.4, 0.9))
    A = rng.normal(size=(3, 3)) * 0.05
    Lam = T0 * (np.eye(3) * rng.uniform(0.9, 1.1) + 0.5 * (A + A.T))
    f = O.target(rng.uniform(0.8, 1.2), rng.uniform(-0.05, 0.05, 3), Lam)
    R = T0 * rng.uniform(0.85, 1.15)
    g, Er, (rho, u, T, sigma, theta) = _g_from_f(P, f, R, c)
    m = O.point_moments(P, g, Er)
    assert abs(m["rho"] - rho) < 1e-14
    np.testing.assert_allclose(m["u"], u, atol=1e-15)
    assert abs(m["T"] - T) < 1e-15
    assert abs(m["R"] - R) < 1e-15
    assert abs(m["theta"] - theta) < 1e-15
    np.testing.assert_allclose(m["sigma"], sigma, atol=1e-15)
    np.testing.assert_allclose(O.point_f(P, g, Er), f, atol=1e-15)
    # the paper's printed relation for theta_T(g)
    a = P.delta * DT / (2 * P.tau1 * (3 + P.delta))
    assert abs(m["thetaTg"] - (T + a * (T - R))) < 1e-15


def test_point_init_round_trip():
    P = _params()
    u = np.array([0.02, -0.03, 0.01])
    g, Er = O.point_init(P, 1.07, u, 0.93 * T0, 1.08 * T0)
    m = O.point_moments(P, g, Er)
    assert abs(m["rho"] - 1.07) < 1e-14
    np.testing.assert_allclose(m["u"], u, atol=1e-15)
    assert abs(m["T"] - 0.93 * T0) < 1e-15
    assert abs(m["R"] - 1.08 * T0) < 1e-15
    np.testing.assert_allclose(m["sigma"], 0.0, atol=1e-15)


@pytest.mark.parametrize("b", [-0.4, 0.0, 0.7])
def test_zero_of_collision(b):
    """f = f^MB with theta_T = theta_R = theta is unchanged (Sec. 4)."""
    P = _params(b=b)
    g, Er = O.point_init(P, 0.96, np.array([0.04, 0.0, -0.02]), 1.05 * T0, 1.05 * T0)
    g2, Er2 = O.point_collide(P, g, Er)
    np.testing.assert_allclose(g2, g, atol=2e-16)
    assert abs(Er2 - Er) < 1e-16


@pytest.mark.parametrize("seed", range(3))
def test_collision_conserves_mass_momentum_total_energy(seed):
    rng = np.random.default_rng(10 + seed)
    c, w = O.lattice()
    P = _params(tau=rng.uniform(0.3, 3), tau1=rng.uniform(0.3, 3), b=rng.uniform(-0.4, 0.9))
    A = rng.normal(size=(3, 3)) * 0.05
    f = O.target(1.0, rng.uniform(-0.05, 0.05, 3), T0 * (np.eye(3) + 0.5 * (A + A.T)))
    g, Er, _ = _g_from_f(P, f, 0.9 * T0, c)
    g2, Er2 = O.point_collide(P, g, Er)
    c2 = (c ** 2).sum(1)
    assert abs(g2.sum() - g.sum()) < 1e-15
    np.testing.assert_allclose(g2 @ c, g @ c, atol=1e-16)
    assert abs((0.5 * g2 @ c2 + Er2) - (0.5 * g @ c2 + Er)) < 1e-15


@pytest.mark.parametrize("tau,tau1,b", [(0.4, 0.3, 0.0), (2.0, 5.0, 0.5), (0.9, 1.7, -0.3)])
def test_homogeneous_relaxation_closed_form(tau, tau1, b):
    """A spatially uniform state relaxes as the trapezoid rule applied to
    d(T - R)/dt = -(T - R)/tau1 and d sigma/dt = -(B - b) sigma / tau
    (B = 1 + tau/tau1), while rho, u and theta stay fixed: on the discrete
    scheme these are exact per step factors."""
    c, w = O.lattice()
    P = O.make_params(2.0, tau, tau1, b, 0.0, DT, 1, 0)
    A = np.array([[0.05, 0.02, -0.01], [0.02, -0.03, 0.015], [-0.01, 0.015, -0.02]])
    f = O.target(1.0, np.array([0.03, -0.01, 0.02]), T0 * (1.02 * np.eye(3) + A))
    g, Er, (rho, u, T, sigma, theta) = _g_from_f(P, f, 0.9 * T0, c)
    S = O.State(P, 1, 1, 1)
    S.g[:] = g
    S.Er[:] = Er
    S.uprev[:] = np.repeat(u, 2)
    r1 = (1 - DT / (2 * tau1)) / (1 + DT / (2 * tau1))
    B = 1 + tau / tau1
    r2 = (1 - DT * (B - b) / (2 * tau)) / (1 + DT * (B - b) / (2 * tau))
    D0 = T - 0.9 * T0
    for n in range(1, 9):
        S.step(1)
        m = O.point_moments(P, S.g[0], S.Er[0])
        assert abs(m["rho"] - rho) < 1e-14
        np.testing.assert_allclose(m["u"], u, atol=1e-15)
        assert abs(m["theta"] - theta) < 1e-14
        assert abs((m["T"] - m["R"]) - D0 * r1 ** n) < 1e-14
        np.testing.assert_allclose(m["sigma"], sigma * r2 ** n, atol=1e-14)


@pytest.mark.parametrize("tau,tau1,b", [(1.0, 1.5, 0.0), (2.0, 3.0, 0.5), (1.2, 1.0, -0.3),
                                        (5.0, 5.0, 0.9)])
def test_h1_non_increasing_in_homogeneous_relaxation(tau, tau1, b):
    """H1 = sum f ln(f/w) - f - (delta/2) rho ln theta_R (Sec. 4, k = -delta/2)
    does not grow while an anisotropic state with theta_T != theta_R relaxes.
    Checked where the trapezoid does not over-relax (tau*, tau1 >= dt/2); with
    tau* < dt/2 the discrete map overshoots and H1 may rise transiently."""
    c, w = O.lattice()
    P = O.make_params(2.0, tau, tau1, b, 0.5, DT, 1, 0)
    Lam = T0 * (np.diag([1.08, 0.95, 0.97]) + 0.02 * (np.ones((3, 3)) - np.eye(3)))
    f = O.target(1.0, np.array([0.03, -0.01, 0.02]), Lam)
    g, Er, _ = _g_from_f(P, f, 0.9 * T0, c)
    S = O.State(P, 1, 1, 1)
    S.g[:] = g
    S.Er[:] = Er
    H = [S.diag()["H1"]]
    for _ in range(40):
        S.step(1)
        H.append(S.diag()["H1"])
    H = np.array(H)
    assert np.all(np.isfinite(H))
    assert np.all(np.diff(H) <= 1e-13 * abs(H[0]))
    assert H[-1] < H[0]


@pytest.mark.parametrize("rho,theta", [(1.0, T0), (1.3, T0), (0.7, 1.1 * T0)])
def test_h1_value_at_rest_equilibrium(rho, theta):
    """At rest with theta_T = theta_R = theta0 the discrete state is f = rho w,
    so H1 = rho ln rho - rho - (delta/2) rho ln theta0 per point; away from
    theta0 compare with the same sum taken over the target itself."""
    P = _params()
    S = O.State(P, 1, 1, 1)
    u0 = np.zeros((3, 2))
    S.init_fields(np.full(2, rho), u0, np.full(2, theta), np.full(2, theta))
    H = S.diag()["H1"]
    c, w = O.lattice()
    feq = O.target(rho, np.zeros(3), theta * np.eye(3))
    expect = 2 * ((feq * np.log(feq / w) - feq).sum() - 0.5 * P.delta * rho * np.log(theta))
    assert abs(H - expect) < 1e-13 * max(1.0, abs(expect))
    if theta == T0:
        closed = 2 * (rho * np.log(rho) - rho - 0.5 * P.delta * rho * np.log(T0))
        assert abs(H - closed) < 1e-13 * max(1.0, abs(closed))
