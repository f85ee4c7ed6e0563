"""Pins of the oracle's lattice and discrete targets against mathematics the
paper fixes: the RD3Q41 isotropy (Sec. 5, Table 1) and the moments of a
Gaussian with mean u and covariance Lambda (Sec. 2, eq. lambdaij)."""
import itertools

import numpy as np
import pytest

import oracle as O

T0 = O.THETA0


def test_theta0_matches_table_caption():
    assert O.theta0() == 0.2948964908710633


def test_velocity_set_shells_and_symmetry():
    c, w = O.lattice()
    assert c.shape == (41, 3)
    # shells by |c|^2: rest, |c|=1 axis, (1,1,0), (1/2)^3, (1,1,1), |c|=2 axis
    c2 = np.round((c ** 2).sum(1), 12)
    counts = {v: int((c2 == v).sum()) for v in np.unique(c2)}
    assert counts == {0.0: 1, 0.75: 8, 1.0: 6, 2.0: 12, 3.0: 8, 4.0: 6}
    # closed under negation and all distinct
    keys = {tuple(v) for v in np.round(c, 12)}
    assert len(keys) == 41
    assert all(tuple(-np.array(k) + 0.0) in keys for k in keys)
    # half-integer velocities have all three components +-1/2
    half = np.abs(c) == 0.5
    assert np.all(half.sum(1)[half.any(1)] == 3)


def test_weights_positive_and_normalised():
    c, w = O.lattice()
    assert w.min() > 0.0
    assert abs(w.sum() - 1.0) < 1e-15


def _moment(w, c, powers):
    m = w.copy()
    for a, p in enumerate(powers):
        m = m * c[:, a] ** p
    return m.sum()


def test_isotropy_up_to_fourth_order_and_contracted_sixth():
    c, w = O.lattice()
    # odd moments vanish
    for powers in itertools.product(range(4), repeat=3):
        if sum(powers) % 2 == 1 and sum(powers) <= 5:
            assert abs(_moment(w, c, powers)) < 1e-15
    # second order: theta0 delta_ab
    assert abs(_moment(w, c, (2, 0, 0)) - T0) < 1e-15
    assert abs(_moment(w, c, (1, 1, 0))) < 1e-15
    # fourth order: theta0^2 (d_ab d_cd + d_ac d_bd + d_ad d_bc)
    assert abs(_moment(w, c, (4, 0, 0)) - 3 * T0 ** 2) < 1e-15
    assert abs(_moment(w, c, (2, 2, 0)) - T0 ** 2) < 1e-15
    assert abs(_moment(w, c, (0, 2, 2)) - T0 ** 2) < 1e-15
    # contracted sixth order: sum w c^2 c_a c_b c_c c_d = 7 theta0^3 (d d + d d + d d)
    c2 = (c ** 2).sum(1)
    assert abs((w * c2 * c[:, 0] ** 4).sum() - 21 * T0 ** 3) < 1e-14
    assert abs((w * c2 * c[:, 0] ** 2 * c[:, 1] ** 2).sum() - 7 * T0 ** 3) < 1e-14
    # the full sixth order is not isotropic on this lattice (reason the
    # equilibrium stops at third order)
    assert abs(_moment(w, c, (2, 2, 2)) - T0 ** 3) > 0.5 * T0 ** 3


def _random_state(rng, aniso=0.08, umax=0.06):
    rho = rng.uniform(0.8, 1.2)
    u = rng.uniform(-umax, umax, 3)
    A = rng.normal(size=(3, 3)) * aniso
    Lam = T0 * (np.eye(3) * rng.uniform(0.9, 1.1) + 0.5 * (A + A.T))
    return rho, u, Lam


def test_target_reduces_to_weights_at_rest():
    c, w = O.lattice()
    f = O.target(1.3, np.zeros(3), T0 * np.eye(3))
    np.testing.assert_allclose(f, 1.3 * w, rtol=0, atol=1e-16)


@pytest.mark.parametrize("seed", range(5))
def test_target_gaussian_moments(seed):
    """Density, momentum, the full pressure tensor and the energy flux of the
    discrete target equal those of the Gaussian N(u, Lambda) times rho."""
    rng = np.random.default_rng(seed)
    c, w = O.lattice()
    rho, u, Lam = _random_state(rng)
    f = O.target(rho, u, Lam)
    assert abs(f.sum() - rho) < 1e-14
    np.testing.assert_allclose(f @ c, rho * u, atol=1e-15)
    P = np.einsum("i,ia,ib->ab", f, c, c)
    np.testing.assert_allclose(P, rho * (np.outer(u, u) + Lam), atol=1e-15)
    c2 = (c ** 2).sum(1)
    q = (f * c2) @ c
    q_gauss = rho * (u * (u @ u + np.trace(Lam)) + 2.0 * Lam @ u)
    np.testing.assert_allclose(q, q_gauss, atol=1e-15)


def test_target_third_moment_exact_at_linear_order():
    """sum f c_a c_b c_c = rho (u_a Lam_bc + u_b Lam_ca + u_c Lam_ab + u_a u_b u_c)
    holds up to terms quadratic in (u, Lambda - theta0 I)."""
    c, w = O.lattice()
    eps = 1e-4
    rng = np.random.default_rng(7)
    u = eps * rng.normal(size=3)
    Lam = T0 * np.eye(3) + eps * T0 * np.diag(rng.normal(size=3))
    f = O.target(1.0, u, Lam)
    Qm = np.einsum("i,ia,ib,ic->abc", f, c, c, c)
    Qg = (np.einsum("a,bc->abc", u, Lam) + np.einsum("b,ca->abc", u, Lam)
          + np.einsum("c,ab->abc", u, Lam))
    assert np.abs(Qm - Qg).max() < 10 * eps ** 2
