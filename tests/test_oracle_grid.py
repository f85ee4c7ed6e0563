"""Pins of the oracle's grid operations: pull streaming on the BCC lattice
(brute force over physical positions), the MacCormack advection and the FTCS
diffusion of the rotational energy (closed-form amplification factors of the
two schemes, Sec. 5 steps 2 and 3), conservation on a periodic box (Sec. 4,
eq. ConservedMomEq), translation invariance and the x-reservoir boundary."""
import numpy as np
import pytest

import oracle as O
import rpk_inputs as I

T0 = O.THETA0
INF = 1e300  # relaxation time that switches a collision term off exactly


def _positions2(nx, ny, nz):
    """Doubled physical coordinates of every point, as integer tuples."""
    X = I.positions(nx, ny, nz)
    return [tuple(int(round(2 * v)) for v in X[:, p]) for p in range(X.shape[1])]


@pytest.mark.parametrize("dims", [(5, 4, 3), (2, 1, 1), (3, 2, 1), (1, 1, 1)])
def test_pull_streaming_matches_positions(dims):
    """With both relaxation times infinite the step is pure streaming: the
    population i at position r comes from position r - c_i (periodic)."""
    nx, ny, nz = dims
    P = O.make_params(2.0, INF, INF, 0.0, 0.0, 1.0, 1, 0)
    S = O.State(P, nx, ny, nz)
    rng = np.random.default_rng(3)
    c, w = O.lattice()
    S.g[:] = w[None, :] * rng.uniform(0.5, 1.5, size=S.g.shape)
    S.Er[:] = T0
    g0 = S.g.copy()
    S.step(1)
    pos = _positions2(nx, ny, nz)
    L2 = np.array([2 * nx, 2 * ny, 2 * nz])
    where = {p: k for k, p in enumerate(pos)}
    expected = np.empty_like(g0)
    for k, p in enumerate(pos):
        for i in range(41):
            src = tuple(int(v) for v in np.mod(np.array(p) - np.round(2 * c[i]).astype(int), L2))
            expected[k, i] = g0[where[src], i]
    np.testing.assert_array_equal(S.g, expected)


def _advect_setup(nx, ny, nz, U, amp, axis, mode=1):
    P = O.make_params(2.0, INF, INF, 0.0, 0.0, 1.0, 1, 0)
    f = I.uniform(nx, ny, nz, T0, u=U)
    S = O.State(P, nx, ny, nz).init_fields(f["rho"], f["u"], f["T"], f["R"])
    X = I.positions(nx, ny, nz)
    n = (nx, ny, nz)[axis]
    k = 2 * np.pi * mode / n
    base = S.Er.copy()
    S.Er[:] = base * (1.0 + amp * np.cos(k * X[axis]))
    return S, X, k, base


@pytest.mark.parametrize("axis,Ucomp", [(0, 0.31), (1, -0.22), (2, 0.17)])
def test_maccormack_amplification(axis, Ucomp):
    """Constant velocity, uniform density: the predictor/corrector pair is the
    Lax-Wendroff scheme, amplification 1 - i C sin k - C^2 (1 - cos k)."""
    dims = [1, 1, 1]
    dims[axis] = 12
    U = [0.0, 0.0, 0.0]
    U[axis] = Ucomp
    S, X, k, base = _advect_setup(*dims, U, 1e-3, axis)
    nsteps = 7
    S.step(nsteps)
    C = Ucomp
    G = 1 - 1j * C * np.sin(k) - C ** 2 * (1 - np.cos(k))
    expected = base * (1.0 + 1e-3 * np.real(G ** nsteps * np.exp(1j * k * X[axis])))
    np.testing.assert_allclose(S.Er, expected, rtol=0, atol=1e-15)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_ftcs_amplification(axis):
    """Zero velocity, tau1 infinite (no exchange), kappa_R > 0: each FTCS
    sub-step multiplies a mode by 1 - h D 2 (1 - cos k), h = dt/nsub,
    D = 2 kappa_R/(delta rho), kappa_R = k_r 5 p tau/(2B), B = 1."""
    dims = [1, 1, 1]
    dims[axis] = 10
    tau, kr, nsub = 1.3, 0.6, 3
    P = O.make_params(2.0, tau, INF, 0.0, kr, 1.0, nsub, 0)
    f = I.uniform(*dims, T0)
    S = O.State(P, *dims).init_fields(f["rho"], f["u"], f["T"], f["R"])
    X = I.positions(*dims)
    k = 2 * np.pi / dims[axis]
    eps = 1e-7
    base = S.Er.copy()
    S.Er[:] = base * (1.0 + eps * np.cos(k * X[axis]))
    nsteps = 5
    S.step(nsteps)
    K0 = kr * 5 * 1.0 * T0 * tau / 2
    D = 2 * K0 / (2.0 * 1.0)
    Gs = 1 - (1.0 / nsub) * D * 2 * (1 - np.cos(k))
    expected = base * (1.0 + eps * Gs ** (nsub * nsteps) * np.cos(k * X[axis]))
    np.testing.assert_allclose(S.Er, expected, rtol=0, atol=1e-15)


def test_periodic_conservation_1000_steps():
    """Mass, momentum and total energy E_T + E_R are conserved to round-off on a
    periodic box (Sec. 4, eq. ConservedMomEq); 1000 steps, all terms active."""
    nx, ny, nz = 6, 5, 4
    P = O.make_params(2.0, 0.6, 0.8, 0.4, 0.9, 1.0, 2, 0)
    f = I.random_smooth(nx, ny, nz, T0)
    S = O.State(P, nx, ny, nz).init_fields(f["rho"], f["u"], f["T"], f["R"])
    d0 = S.diag()
    S.step(1000)
    d1 = S.diag()
    M0 = d0["M"]
    assert abs(d1["M"] - M0) < 1e-12 * M0
    assert np.abs(d1["J"] - d0["J"]).max() < 1e-12 * M0
    assert abs(d1["E"] - d0["E"]) < 1e-12 * d0["E"]
    F = S.fields()
    assert np.all(np.isfinite(F["rho"])) and d1["min_g"] > 0


def test_translation_invariance_bitwise():
    nx, ny, nz = 6, 4, 3
    P = O.make_params(2.0, 0.6, 0.8, 0.2, 0.9, 1.0, 2, 0)
    f = I.random_smooth(nx, ny, nz, T0)

    def roll(a):  # shift every field by one cell along +y on both sublattices
        return np.roll(a.reshape(-1, 2, nz, ny, nx), 1, axis=3).reshape(a.shape)

    A = O.State(P, nx, ny, nz).init_fields(f["rho"], f["u"], f["T"], f["R"]).step(20)
    B = O.State(P, nx, ny, nz).init_fields(roll(f["rho"]), roll(f["u"]), roll(f["T"]),
                                             roll(f["R"])).step(20)
    FA, FB = A.fields(), B.fields()
    for key in ("rho", "T", "R"):
        np.testing.assert_array_equal(roll(FA[key]), FB[key])
    np.testing.assert_array_equal(roll(FA["u"]), FB["u"])


def test_reservoirs_leave_the_interior_unchanged():
    """With bcx = 1 the points beyond the reach of the ends (populations move
    at most 2 cells and the transport nsub + 1 cells per step) match the
    periodic run bit for bit."""
    nx, nsteps = 48, 4
    P0 = O.make_params(2.0, 0.7, 0.9, 0.0, 0.5, 1.0, 1, 0)
    P1 = O.make_params(2.0, 0.7, 0.9, 0.0, 0.5, 1.0, 1, 1)
    f, res = I.shock_tube(nx, T0, rho_r=1 / 1.5, p_r=0.5)
    # periodic image of a tube is a second diaphragm at x = 0; keep the probe
    # region around the interior diaphragm only
    A = O.State(P0, nx, 1, 1).init_fields(f["rho"], f["u"], f["T"], f["R"]).step(nsteps)
    B = O.State(P1, nx, 1, 1, reservoirs=res).init_fields(f["rho"], f["u"], f["T"],
                                                          f["R"]).step(nsteps)
    X = I.positions(nx, 1, 1)[0]
    reach = nsteps * 3 + 2
    inner = (X > reach) & (X < nx - 1 - reach)
    np.testing.assert_array_equal(A.g[inner], B.g[inner])
    np.testing.assert_array_equal(A.Er[inner], B.Er[inner])


def test_reservoir_equilibrium_is_fixed():
    nx = 16
    P = O.make_params(2.0, 0.7, 0.9, 0.0, 0.5, 1.0, 1, 1)
    f = I.uniform(nx, 1, 1, T0, rho=0.8, T=1.1 * T0)
    res = np.array([0.8, 0, 0, 0, 1.1 * T0, 1.1 * T0] * 2)
    S = O.State(P, nx, 1, 1, reservoirs=res).init_fields(f["rho"], f["u"], f["T"], f["R"])
    g0, E0 = S.g.copy(), S.Er.copy()
    S.step(10)
    np.testing.assert_allclose(S.g, g0, atol=1e-16)
    np.testing.assert_allclose(S.Er, E0, atol=1e-16)


def test_one_step_from_rest_is_mirror_symmetric():
    """x -> -x symmetry of one step from a state at rest with varying rho,
    theta_T and theta_R (no advection at u = 0): pins the streaming of the
    half velocities and the symmetric face conductivity of the FTCS."""
    from test_oracle_mutants import _pin_mirror
    assert _pin_mirror()
