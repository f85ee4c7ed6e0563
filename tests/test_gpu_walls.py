"""Diffuse walls on the GPU (rpk_set_walls, rpk_set_x_walls) against the FP64
oracle, and the paper's three wall experiments run on the GPU path (Sec. 6).

Parity bars as for the periodic lattice: FP64 relative L-inf <= 1e-12 per
field (rounding order differs), FP32 <= 1e-5 (u on the c_s scale). Sizes span
several 128-point x rows and 8-row y tiles of the transport with ragged tails,
the smallest channel (ny = 2) and single columns (nx = nz = 1); the full-size
case runs a 256 x 32 x 128 channel whose input is an x-z tiling of a 16 x 32 x 8
box, so the exact answer is the oracle's small run tiled back.

E4 (startup Couette flow, Sec. 6): the paper's 128 x 64 x 8 grid, top wall
started impulsively; u(y, t) against the printed series solution at diffusion
times t* = nu t / L^2 = 0.02 ... 0.5.
E5 (conduction in a square cavity, Sec. 6): 128 x 128 cells, walls on all four
sides, the top one hotter by 0.1 theta0;
the steady theta along the paper's lines x = 0.1L, 0.2L, 0.5L and
y = 0.25L, 0.5L, 0.75L against the printed series.
E6 (thermal Couette flow, Sec. 6): 128 points between the walls, walls at
theta0 -+ dT/2, top wall at Mach 0.1, Ec = U0^2/(c_p dT) = 1,
Pr = 0.75, 2.5, 5, 7.5, 10; the steady theta(y) against the printed profile
(T - T0)/dT = y/H + (Pr Ec/2)(y/H)(1 - y/H)."""
import numpy as np
import pytest

import oracle as O
import paper_2201_05280_gb300 as rpk
import rpk_inputs as I

pytestmark = pytest.mark.gpu

T0 = 0.2948964908710633
CS = np.sqrt(1.4 * T0)
WALLS = ([0.03, 0.0, -0.02, T0 * 1.02], [-0.04, 0.0, 0.01, T0 * 0.97])
RELAX = dict(delta=2.0, tau=0.6, tau1=0.8, b=0.3, k_r=0.9, nsub=2)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2201_05280_gb300 import build as B
    B.build()
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


def rel(a, b, floor=1e-300):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), floor))


XWALLS = ([0.0, 0.02, -0.01, T0 * 1.02], [0.0, -0.03, 0.02, T0 * 0.98])


def run_pair(nx, ny, nz, f, relax, nsteps, precision="f64", walls=WALLS, xwalls=None):
    lat = rpk.Lattice(nx, ny, nz, precision=precision).set_relax(**relax)
    if walls is not None:
        lat.set_walls(*walls)
    if xwalls is not None:
        lat.set_x_walls(*xwalls)
    lat.init_fields(f["rho"], f["u"], f["T"], f["R"])
    nsub = lat.info()["nsub"]
    P = O.make_params(relax["delta"], relax["tau"], relax["tau1"], relax.get("b", 0.0),
                      relax.get("k_r", 0.0), 1.0, nsub,
                      walls=None if walls is None else list(walls[0]) + list(walls[1]),
                      xwalls=None if xwalls is None else list(xwalls[0]) + list(xwalls[1]))
    S = O.State(P, nx, ny, nz).init_fields(f["rho"], f["u"], f["T"], f["R"])
    lat.step(nsteps)
    S.step(nsteps)
    return lat.read_moments(), S.fields(), lat, S


def check(got, ref, tol, keys=("rho", "u", "T", "R", "Erot")):
    errs = {k: rel(got[k], ref[k], CS if k == "u" else 1e-300) for k in keys}
    assert all(v <= tol for v in errs.values()), errs
    return errs


@pytest.mark.parametrize("dims", [(150, 10, 3), (5, 2, 3), (1, 16, 1), (33, 9, 1)])
def test_f64_parity_with_walls(dims):
    nx, ny, nz = dims
    f = I.random_smooth(nx, ny, nz, T0, seed=21)
    got, ref, lat, S = run_pair(nx, ny, nz, f, RELAX, 40)
    check(got, ref, 1e-12)
    d, dr = lat.diagnostics(), S.diag()
    assert abs(d["M"] - dr["M"]) <= 1e-12 * dr["M"]
    assert abs(d["E"] - dr["E"]) <= 1e-12 * dr["E"]
    assert d["status"] == 0


@pytest.mark.parametrize("dims", [(12, 7, 3), (2, 5, 2), (137, 3, 2)])
def test_f64_parity_with_x_walls(dims):
    nx, ny, nz = dims
    f = I.random_smooth(nx, ny, nz, T0, seed=31)
    got, ref, lat, S = run_pair(nx, ny, nz, f, RELAX, 40, walls=None, xwalls=XWALLS)
    check(got, ref, 1e-12)
    assert abs(lat.diagnostics()["M"] - S.diag()["M"]) <= 1e-12 * S.diag()["M"]


@pytest.mark.parametrize("dims", [(9, 10, 2), (130, 6, 1), (2, 2, 2)])
def test_f64_parity_with_walls_on_x_and_y(dims):
    nx, ny, nz = dims
    f = I.random_smooth(nx, ny, nz, T0, seed=32)
    got, ref, lat, S = run_pair(nx, ny, nz, f, RELAX, 40, xwalls=XWALLS)
    check(got, ref, 1e-12)
    d, dr = lat.diagnostics(), S.diag()
    assert abs(d["M"] - dr["M"]) <= 1e-12 * dr["M"]
    assert abs(d["E"] - dr["E"]) <= 1e-12 * dr["E"]
    assert d["status"] == 0


def test_f32_parity_with_walls_on_x_and_y():
    nx, ny, nz = 24, 20, 3
    f = I.random_smooth(nx, ny, nz, T0, seed=33, amp=2e-3, aniso_R=2e-3)
    got, ref, _, _ = run_pair(nx, ny, nz, f, RELAX, 300, precision="f32", xwalls=XWALLS)
    check(got, ref, 1e-5, keys=("rho", "u", "T", "Erot"))


def test_four_walls_fixed_point_mass_and_checkpoint(tmp_path):
    u = [0.0, 0.0, 0.03]
    w = u + [0.31]
    lat = rpk.Lattice(5, 4, 3, precision="f64").set_relax(**RELAX).set_walls(w, w).set_x_walls(w, w)
    f = I.uniform(5, 4, 3, 0.31, rho=1.1, u=u)
    lat.init_fields(f["rho"], f["u"], f["T"], f["R"])
    a = lat.read_moments()
    lat.step(7)
    b = lat.read_moments()
    for k in ("rho", "u", "T", "R"):
        assert np.abs(b[k] - a[k]).max() < 1e-13, k
    nx, ny, nz = 12, 10, 4
    f = I.random_smooth(nx, ny, nz, T0, seed=34)
    lat = rpk.Lattice(nx, ny, nz, precision="f64").set_relax(**RELAX)
    lat.set_walls(*WALLS).set_x_walls(*XWALLS)
    lat.init_fields(f["rho"], f["u"], f["T"], f["R"])
    m0 = lat.diagnostics()["M"]
    lat.step(1000)
    assert abs(lat.diagnostics()["M"] - m0) <= 1e-12 * m0
    path = str(tmp_path / "four.ckpt")
    lat.save(path)
    lat.step(9)
    other = rpk.Lattice(nx, ny, nz, precision="f64")
    other.load(path)
    other.step(9)
    ma, mb = lat.read_moments(), other.read_moments()
    for k in ("rho", "u", "T", "R"):
        assert np.array_equal(ma[k], mb[k]), k


@pytest.mark.parametrize("dims,axes", [((10, 7, 2), "y"), ((7, 3, 2), "x"), ((9, 6, 2), "xy")])
def test_f64_parity_paper_mode_between_walls(dims, axes):
    """The paper's theta_R solver (Sec. 5) between diffuse walls: the wall
    ghosts of its advection differences and Laplacian against the oracle."""
    nx, ny, nz = dims
    f = I.random_smooth(nx, ny, nz, T0, seed=35)
    walls = WALLS if "y" in axes else None
    xwalls = XWALLS if "x" in axes else None
    lat = rpk.Lattice(nx, ny, nz, precision="f64").set_relax(**RELAX).set_rot_mode("paper")
    if walls:
        lat.set_walls(*walls)
    if xwalls:
        lat.set_x_walls(*xwalls)
    lat.init_fields(f["rho"], f["u"], f["T"], f["R"]).step(30)
    P = O.make_params(2.0, 0.6, 0.8, 0.3, 0.9, 1.0, 2, rot_mode=1,
                      walls=None if walls is None else list(walls[0]) + list(walls[1]),
                      xwalls=None if xwalls is None else list(xwalls[0]) + list(xwalls[1]))
    S = O.State(P, nx, ny, nz).init_fields(f["rho"], f["u"], f["T"], f["R"]).step(30)
    check(lat.read_moments(), S.fields(), 1e-12)
    d = lat.diagnostics()
    assert abs(d["M"] - S.diag()["M"]) <= 1e-12 * S.diag()["M"] and d["status"] == 0


def test_f64_parity_with_walls_auto_nsub_and_strong_rotational_conduction():
    # k_r = 2 at tau = 0.9: nsub chosen by the library for the near-wall faces
    relax = dict(delta=2.0, tau=0.9, tau1=1.5, b=-0.2, k_r=2.0)
    nx, ny, nz = 12, 12, 2
    f = I.random_smooth(nx, ny, nz, T0, seed=22)
    got, ref, lat, S = run_pair(nx, ny, nz, f, relax, 60)
    assert lat.info()["nsub"] >= 2
    check(got, ref, 1e-12)


def test_f32_parity_with_walls():
    nx, ny, nz = 40, 24, 2
    f = I.random_smooth(nx, ny, nz, T0, seed=23, amp=2e-3, aniso_R=2e-3)
    got, ref, _, _ = run_pair(nx, ny, nz, f, RELAX, 300, precision="f32")
    check(got, ref, 1e-5, keys=("rho", "u", "T", "Erot"))


def test_f64_walls_conserve_mass_1000_steps():
    nx, ny, nz = 16, 8, 6
    f = I.random_smooth(nx, ny, nz, T0, seed=24)
    lat = rpk.Lattice(nx, ny, nz, precision="f64").set_relax(**RELAX).set_walls(*WALLS)
    lat.init_fields(f["rho"], f["u"], f["T"], f["R"])
    d0 = lat.diagnostics()
    lat.step(1000)
    d1 = lat.diagnostics()
    assert abs(d1["M"] - d0["M"]) <= 1e-12 * d0["M"]
    assert d1["status"] == 0


def test_state_equal_to_both_walls_is_fixed():
    u = np.array([0.05, 0.0, 0.02])
    w = list(u) + [0.31]
    lat = rpk.Lattice(6, 4, 3, precision="f64").set_relax(**RELAX).set_walls(w, w)
    f = I.uniform(6, 4, 3, 0.31, rho=1.1, u=u)
    lat.init_fields(f["rho"], f["u"], f["T"], f["R"])
    a = lat.read_moments()
    lat.step(7)
    b = lat.read_moments()
    for k in ("rho", "u", "T", "R"):
        assert np.abs(b[k] - a[k]).max() < 1e-13, k


def test_full_size_channel_f32_against_tiled_oracle():
    small = (16, 32, 8)
    reps = (16, 1, 16)
    nsteps = 50
    f = I.random_smooth(*small, T0, seed=25, amp=2e-3, aniso_R=2e-3)
    F = I.tile(f, *small, reps)
    nx, ny, nz = (small[0] * reps[0], small[1], small[2] * reps[2])
    lat = rpk.Lattice(nx, ny, nz, precision="f32").set_relax(**RELAX).set_walls(*WALLS)
    lat.init_fields(F["rho"], F["u"], F["T"], F["R"])
    lat.step(nsteps)
    got = lat.read_moments()
    d = lat.diagnostics()
    lat.close()
    P = O.make_params(2.0, 0.6, 0.8, 0.3, 0.9, 1.0, 2, walls=list(WALLS[0]) + list(WALLS[1]))
    Fs = O.State(P, *small).init_fields(f["rho"], f["u"], f["T"], f["R"]).step(nsteps).fields()
    ref = I.tile(Fs, *small, reps)
    ref["Erot"] = I.tile(dict(Fs, rho=Fs["Erot"]), *small, reps)["rho"]
    check(got, ref, 1e-5, keys=("rho", "u", "T", "Erot"))
    assert d["status"] == 0


def test_checkpoint_with_walls_is_bitwise(tmp_path):
    nx, ny, nz = 10, 6, 2
    f = I.random_smooth(nx, ny, nz, T0, seed=26)
    a = rpk.Lattice(nx, ny, nz, precision="f32").set_relax(**RELAX).set_walls(*WALLS)
    a.init_fields(f["rho"], f["u"], f["T"], f["R"]).step(10)
    path = str(tmp_path / "walls.ckpt")
    a.save(path)
    a.step(15)
    b = rpk.Lattice(nx, ny, nz, precision="f32")
    b.load(path)
    b.step(15)
    ma, mb = a.read_moments(), b.read_moments()
    for k in ("rho", "u", "T", "R"):
        assert np.array_equal(ma[k], mb[k]), k


def test_wall_argument_errors():
    with pytest.raises(rpk.RpkError):
        rpk.Lattice(4, 1, 2).set_relax(**RELAX).set_walls(*WALLS)          # ny < 2
    with pytest.raises(rpk.RpkError):
        rpk.Lattice(4, 4, 2, bc_x="reservoir").set_relax(**RELAX).set_walls(*WALLS)
    lat = rpk.Lattice(4, 4, 2).set_relax(**RELAX)
    with pytest.raises(rpk.RpkError):
        lat.set_walls([0, 0.01, 0, T0], [0, 0, 0, T0])                    # normal velocity
    with pytest.raises(rpk.RpkError):
        lat.set_walls([0, 0, 0, -1.0], [0, 0, 0, T0])                     # theta <= 0
    lat.set_walls(*WALLS)
    lat.set_walls()                                                        # periodic again
    with pytest.raises(rpk.RpkError):
        rpk.Lattice(1, 4, 2).set_relax(**RELAX).set_x_walls(*XWALLS)     # nx < 2
    with pytest.raises(rpk.RpkError):
        rpk.Lattice(4, 4, 2, bc_x="reservoir").set_relax(**RELAX).set_x_walls(*XWALLS)
    with pytest.raises(rpk.RpkError):
        rpk.Lattice(4, 4, 2).set_relax(**RELAX).set_x_walls([0.01, 0, 0, T0], [0, 0, 0, T0])


# ---------------------------------------------------------------------------
# E4: startup Couette flow (Sec. 6)


def _series(yL, ts):
    k = np.arange(1, 2000)[:, None]
    return yL - (2 / np.pi) * np.sum(np.exp(-(k * np.pi) ** 2 * ts) / k * np.sin(k * np.pi * (1 - yL)),
                                     axis=0)


def test_e4_startup_couette_follows_the_series_solution():
    nx, ny, nz = 128, 64, 8
    nu, U = 0.1, 0.1 * CS
    eta, etaB, kap = rpk.gas_from_nondim(1.4, nu, 0.6, 0.71)
    lat = rpk.Lattice(nx, ny, nz, precision="f32").set_gas(1.4, eta, etaB, kap)
    lat.set_walls([0, 0, 0, T0], [U, 0, 0, T0])
    f = I.uniform(nx, ny, nz, T0)
    lat.init_fields(f["rho"], f["u"], f["T"], f["R"])
    y = I.positions(nx, ny, nz)[1] + 0.25
    L = ny
    errs = {}
    for ts in (0.02, 0.05, 0.1, 0.2, 0.5):
        lat.step(int(round(ts * L * L / nu)) - lat.info()["steps"])
        u = lat.read_moments()["u"][0] / U
        errs[ts] = float(np.abs(u - _series(y / L, lat.info()["steps"] * nu / L ** 2)).max())
    print("E4 max |u/U - series| by t*:", errs)
    assert max(errs.values()) < 0.02, errs
    assert lat.diagnostics()["status"] == 0


# ---------------------------------------------------------------------------
# E6: thermal Couette flow (Sec. 6)


def _relax_for_pr(Pr, nu):
    """tau1 = 8 tau (B = 9/8, the bulk viscosity plays no part in plane
    Couette flow); Pr > 7/5 through the ES parameter b = B (1 - 7/(5 Pr)) with
    k_r = 0, Pr <= 7/5 through k_r = 7/(5 Pr) - 1 with b = 0 (Sec. 4:
    Pr = (B/(B - b))(1 + delta/5)/(1 + k_r)); eta = p tau/(B - b) = nu."""
    B = 1.125
    b, kr = (B * (1 - 1.4 / Pr), 0.0) if Pr > 1.4 else (0.0, 1.4 / Pr - 1)
    tau = nu * (B - b) / T0
    return dict(delta=2.0, tau=tau, tau1=8 * tau, b=b, k_r=kr)


@pytest.mark.parametrize("Pr", [0.75, 2.5, 5.0, 7.5, 10.0])
def test_e6_thermal_couette_profile(Pr):
    ny, nu = 64, 0.2
    U0 = 0.1 * CS
    dT = U0 ** 2 / 3.5  # Ec = 1, c_p = 7/2
    lat = rpk.Lattice(1, ny, 1, precision="f64").set_relax(**_relax_for_pr(Pr, nu))
    lat.set_walls([0, 0, 0, T0 - dT / 2], [U0, 0, 0, T0 + dT / 2])
    f = I.uniform(1, ny, 1, T0)
    lat.init_fields(f["rho"], f["u"], f["T"], f["R"])
    H = ny
    lat.step(int(1.2 * H * H / (nu / Pr)))
    m = lat.read_moments()
    th = (3 * m["T"] + 2 * m["R"]) / 5
    eta = (I.positions(1, ny, 1)[1] + 0.25) / H
    exact = eta + 0.5 * Pr * eta * (1 - eta)
    got = (th - (T0 - dT / 2)) / dT
    err = float(np.abs(got - exact).max() / exact.max())
    print("E6 Pr %g: max |theta - exact| / max exact = %.4f" % (Pr, err))
    assert err < 0.03, (Pr, err)
    assert lat.diagnostics()["status"] == 0


# ---------------------------------------------------------------------------
# E5: conduction in a square cavity heated from the top (Sec. 6)


def _cavity_series(xi, eta, nmax=399):
    """(T - T0)/(T1 - T0) = (2/pi) sum_n ((-1)^(n+1) + 1)/n sin(n pi xi)
    sinh(n pi eta)/sinh(n pi) (Sec. 6), the sinh ratio written with
    exponentials."""
    n = np.arange(1, nmax + 1, 2)[:, None]  # only odd n contribute (factor 2)
    ratio = np.exp(n * np.pi * (eta - 1)) * (1 - np.exp(-2 * n * np.pi * eta)) / (1 - np.exp(-2 * n * np.pi))
    return (2 / np.pi) * np.sum(2.0 / n * np.sin(n * np.pi * xi) * ratio, axis=0)


def test_e5_heated_cavity_conduction_follows_the_series_solution():
    n, nu, Pr = 128, 0.2, 0.71
    dT = 0.1 * T0
    eta_, etaB, kap = rpk.gas_from_nondim(1.4, nu, 0.6, Pr)
    lat = rpk.Lattice(n, n, 1, precision="f32").set_gas(1.4, eta_, etaB, kap)
    cold = [0.0, 0.0, 0.0, T0]
    lat.set_walls(cold, [0.0, 0.0, 0.0, T0 + dT]).set_x_walls(cold, cold)
    f = I.uniform(n, n, 1, T0)
    lat.init_fields(f["rho"], f["u"], f["T"], f["R"])
    lat.step(int(0.8 * n * n / (nu / Pr)))
    m = lat.read_moments()
    th = (3 * m["T"] + 2 * m["R"]) / 5
    X = I.positions(n, n, 1)
    xi, eta = (X[0] + 0.25) / n, (X[1] + 0.25) / n
    got = (th - T0) / dT
    ref = _cavity_series(xi, eta)
    lines = (("x=0.1L", np.abs(xi - 0.1) < 0.5 / n), ("x=0.2L", np.abs(xi - 0.2) < 0.5 / n),
             ("x=0.5L", np.abs(xi - 0.5) < 0.5 / n), ("y=0.25L", np.abs(eta - 0.25) < 0.5 / n),
             ("y=0.5L", np.abs(eta - 0.5) < 0.5 / n), ("y=0.75L", np.abs(eta - 0.75) < 0.5 / n))
    full, away = {}, {}
    for name, sel in lines:
        assert sel.sum() >= n // 2, name
        full[name] = float(np.abs(got[sel] - ref[sel]).max())
        sel = sel & (eta <= 0.9)
        away[name] = float(np.abs(got[sel] - ref[sel]).max())
    umax = float(np.abs(m["u"]).max())
    print("E5 max |(T - T0)/dT - series| along the paper's lines:", full,
          "; below 0.9 L:", away, "; max |u| / c_s = %.2e" % (umax / CS))
    # Measured: 1.4% of dT below 0.9 L and 1.75% on the full lines (x = 0.1L,
    # next to the hot corner). The series is the linear, continuum answer. Two
    # effects separate the lattice gas from it: (i) the lattice conductivity
    # depends on theta at O(theta - theta0) (the third-order equilibrium's
    # energy flux is exact only to first order in theta - theta0), so with
    # dT = 0.1 theta0 the profile bends away from the harmonic one -- with dT =
    # 0.01 theta0 the FP64 oracle's interior error at 32 x 32 falls from 1-2% to
    # below 0.5%; (ii) next to the heated wall and its singular corners the gas
    # stays colder than the wall (the oracle at 32 x 32: -1.5% at 0.9 L and
    # -4.4% at 0.96 L on x = 0.1L), shrinking with L. The thermal creep along
    # the walls near the corners stays below 1% of c_s.
    assert max(away.values()) < 0.02, away
    assert max(full.values()) < 0.025, full
    assert umax < 1e-2 * CS
    assert lat.diagnostics()["status"] == 0
