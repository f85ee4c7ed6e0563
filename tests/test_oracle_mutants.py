"""Mutation check of the pins: plausible mistakes are planted in copies of the
oracle source (compiled on the CPU, never used elsewhere) and each must fail at
least one quick pin. This shows the pins constrain every part of the oracle:
lattice weights, the Hermite targets, the g/f recovery, the collision and the
exchange, streaming, MacCormack, FTCS, the time-centred advection velocity,
initialisation and the H function."""
import numpy as np
import pytest

import oracle as O
import rpk_inputs as I
from oracle import params as PM

T0 = O.THETA0

# (name, exact original text, planted mistake)
MUTANTS = [
    ("weight of the (1,1,0) shell", "t * (45.0 * t - 6.0 - 77.0 * t * t) / 26.0",
     "t * (54.0 * t - 6.0 - 77.0 * t * t) / 26.0"),
    ("dropped A3 term", "D[b][c] * u[a] + D[c][a] * u[b]);", "D[c][a] * u[b]);"),
    ("second-order Hermite factor", "h2 / (2.0 * t0 * t0)", "h2 / (t0 * t0)"),
    ("third-order Hermite factor", "h3 / (6.0 * t0 * t0 * t0)", "h3 / (2.0 * t0 * t0 * t0)"),
    ("theta_T(g) without -rho u^2", "m->thetaTg = (trP - rho * u2)", "m->thetaTg = (trP)"),
    ("wrong sign in the theta_T(g) relation",
     "a_ = P->delta * P->dt / (2.0 * P->tau1 * (3.0 + P->delta));",
     "a_ = -P->delta * P->dt / (2.0 * P->tau1 * (3.0 + P->delta));"),
    ("transposed Cramer numerator", "m->R = ((1.0 + a_) * Rt + X * m->thetaTg) / det;",
     "m->R = ((1.0 + X) * Rt + a_ * m->thetaTg) / det;"),
    ("sign of b in the stress factor", "- P->b * P->dt / (2.0 * P->tau)",
     "+ P->b * P->dt / (2.0 * P->tau)"),
    ("relaxation weight", "(1.0 - 2.0 * bs) * g[i]", "(1.0 - bs) * g[i]"),
    ("exchange sign", "(m.theta - m.R) / P->tau1;", "(m.R - m.theta) / P->tau1;"),
    ("streaming direction", "int pos2 = 2 * idx[a] + s - (int)lround(2.0 * C[i][a]);",
     "int pos2 = 2 * idx[a] + s + (int)lround(2.0 * C[i][a]);"),
    ("predictor with backward differences", "long q = axis_nb(P, &G, p, a, +1);",
     "long q = axis_nb(P, &G, p, a, -1);"),
    ("advection with u(t) instead of the centred velocity",
     "v[p] = 1.5 * u[p] - 0.5 * uprev[p];", "v[p] = u[p];"),
    ("one-sided face conductivity",
     "acc += 0.5 * (kap[p] + kp) * (thp - th[p]) - 0.5 * (kap[p] + km) * (th[p] - thm);",
     "acc += kp * (thp - th[p]) - kap[p] * (th[p] - thm);"),
    ("H without the weights", "Hp += f[i] * log(f[i] / W[i]) - f[i];",
     "Hp += f[i] * log(f[i]) - f[i];"),
    ("initial E_R shift sign", "*Er = 0.5 * P->delta * rho * R -", "*Er = 0.5 * P->delta * rho * R +"),
]


def _pin_targets():
    c, w = O.lattice()
    if abs(w.sum() - 1) > 1e-14 or abs((w * c[:, 0] ** 2).sum() - T0) > 1e-14:
        return False
    rng = np.random.default_rng(1)
    u = rng.uniform(-0.05, 0.05, 3)
    A = rng.normal(size=(3, 3)) * 0.05
    Lam = T0 * (np.eye(3) + 0.5 * (A + A.T))
    f = O.target(1.1, u, Lam)
    P = np.einsum("i,ia,ib->ab", f, c, c)
    c2 = (c ** 2).sum(1)
    q = (f * c2) @ c
    qg = 1.1 * (u * (u @ u + np.trace(Lam)) + 2 * Lam @ u)
    return (abs(f.sum() - 1.1) < 1e-13 and np.allclose(f @ c, 1.1 * u, atol=1e-14)
            and np.allclose(P, 1.1 * (np.outer(u, u) + Lam), atol=1e-14)
            and np.allclose(q, qg, atol=1e-14))


def _pin_relaxation():
    """closed-form homogeneous relaxation (exact per step) and recovery."""
    c, w = O.lattice()
    tau, tau1, b = 0.9, 1.7, -0.3
    P = O.make_params(2.0, tau, tau1, b, 0.0, 1.0, 1, 0)
    A = np.array([[0.05, 0.02, -0.01], [0.02, -0.03, 0.015], [-0.01, 0.015, -0.02]])
    f = O.target(1.0, np.array([0.03, -0.01, 0.02]), T0 * (1.02 * np.eye(3) + A))
    rho, u = f.sum(), f @ c / f.sum()
    Pt = np.einsum("i,ia,ib->ab", f, c, c)
    T = (np.trace(Pt) - rho * u @ u) / (3 * rho)
    sig = Pt - rho * np.outer(u, u) - rho * T * np.eye(3)
    R = 0.9 * T0
    th = (3 * T + 2 * R) / 5
    Om = (O.target(rho, u, T * np.eye(3) + b * sig / rho) - f) / tau + (
        O.target(rho, u, th * np.eye(3)) - f) / tau1
    g = f - 0.5 * Om
    Er = rho * R - 0.5 * rho * (th - R) / tau1
    m = O.point_moments(P, g, Er)
    if not (abs(m["T"] - T) < 1e-14 and abs(m["R"] - R) < 1e-14
            and np.allclose(m["sigma"], sig, atol=1e-14)):
        return False
    S = O.State(P, 1, 1, 1)
    S.g[:] = g
    S.Er[:] = Er
    S.uprev[:] = np.repeat(u, 2)
    r1 = (1 - 1 / (2 * tau1)) / (1 + 1 / (2 * tau1))
    B = 1 + tau / tau1
    r2 = (1 - (B - b) / (2 * tau)) / (1 + (B - b) / (2 * tau))
    for n in range(1, 5):
        S.step(1)
        m = O.point_moments(P, S.g[0], S.Er[0])
        if abs((m["T"] - m["R"]) - (T - R) * r1 ** n) > 1e-13:
            return False
        if not np.allclose(m["sigma"], sig * r2 ** n, atol=1e-13):
            return False
    return True


def _pin_init_round_trip():
    P = O.make_params(2.0, 0.7, 0.9, 0.3, 0.5, 1.0, 1, 0)
    g, Er = O.point_init(P, 1.07, np.array([0.02, -0.03, 0.01]), 0.93 * T0, 1.08 * T0)
    m = O.point_moments(P, g, Er)
    return abs(m["T"] - 0.93 * T0) < 1e-14 and abs(m["R"] - 1.08 * T0) < 1e-14


def _pin_streaming():
    nx, ny, nz = 3, 2, 1
    P = O.make_params(2.0, 1e300, 1e300, 0.0, 0.0, 1.0, 1, 0)
    S = O.State(P, nx, ny, nz)
    c, w = O.lattice()
    S.g[:] = w[None, :] * np.random.default_rng(3).uniform(0.5, 1.5, size=S.g.shape)
    S.Er[:] = T0
    g0 = S.g.copy()
    S.step(1)
    X = I.positions(nx, ny, nz)
    pos = [tuple(int(round(2 * v)) for v in X[:, p]) for p in range(X.shape[1])]
    where = {p: k for k, p in enumerate(pos)}
    L2 = np.array([2 * nx, 2 * ny, 2 * nz])
    for k, p in enumerate(pos):
        for i in range(41):
            src = tuple(int(v) for v in np.mod(np.array(p) - np.round(2 * c[i]).astype(int), L2))
            if S.g[k, i] != g0[where[src], i]:
                return False
    return True


def _pin_maccormack():
    nx, Uc = 12, 0.31
    P = O.make_params(2.0, 1e300, 1e300, 0.0, 0.0, 1.0, 1, 0)
    f = I.uniform(nx, 1, 1, T0, u=(Uc, 0, 0))
    S = O.State(P, nx, 1, 1).init_fields(f["rho"], f["u"], f["T"], f["R"])
    X = I.positions(nx, 1, 1)
    k = 2 * np.pi / nx
    base = S.Er.copy()
    S.Er[:] = base * (1 + 1e-3 * np.cos(k * X[0]))
    S.step(5)
    G = 1 - 1j * Uc * np.sin(k) - Uc ** 2 * (1 - np.cos(k))
    return np.allclose(S.Er, base * (1 + 1e-3 * np.real(G ** 5 * np.exp(1j * k * X[0]))),
                       rtol=0, atol=1e-15)


def _pin_conservation():
    P = O.make_params(2.0, 0.6, 0.8, 0.4, 0.9, 1.0, 2, 0)
    f = I.random_smooth(5, 4, 3, T0)
    S = O.State(P, 5, 4, 3).init_fields(f["rho"], f["u"], f["T"], f["R"])
    d0 = S.diag()
    S.step(50)
    d1 = S.diag()
    return (abs(d1["M"] - d0["M"]) < 1e-12 * d0["M"] and abs(d1["E"] - d0["E"]) < 1e-12 * d0["E"]
            and np.abs(d1["J"] - d0["J"]).max() < 1e-12 * d0["M"])


def _pin_h1_rest():
    P = O.make_params(2.0, 0.7, 0.9, 0.3, 0.5, 1.0, 1, 0)
    S = O.State(P, 1, 1, 1).init_fields(np.full(2, 1.3), np.zeros((3, 2)), np.full(2, T0),
                                        np.full(2, T0))
    closed = 2 * (1.3 * np.log(1.3) - 1.3 - 1.3 * np.log(T0))
    return abs(S.diag()["H1"] - closed) < 1e-12


def _pin_acoustic_attenuation():
    """coarse version of the hydrodynamic acoustic pin (5% instead of 1%)."""
    from scipy.optimize import curve_fit
    nx = 64
    eta, etaB, kap = PM.gas_from_nondim(1.4, 0.08, 0.6, 0.71)
    d, tau, tau1, b, kr = PM.relax_from_gas(1.4, eta, etaB, kap, 0.0)
    P = O.make_params(d, tau, tau1, b, kr, 1.0, PM.nsub_for(d, tau, tau1, kr, T0, 1), 0)
    tr = PM.transport(d, tau, tau1, b, kr)
    f, k = I.acoustic_wave(nx, 1, 1, T0, 1.4, amp=1e-4)
    S = O.State(P, nx, 1, 1).init_fields(f["rho"], f["u"], f["T"], f["R"])
    X = I.positions(nx, 1, 1)[0]
    ts, bs = [0.0], [0.0]
    for _ in range(60):
        S.step(10)
        ts.append(S.t)
        bs.append(2 * np.mean(S.fields()["u"][0] * np.sin(k * X)))
    fn = lambda t, A, G, w, ph: A * np.exp(-G * t) * np.sin(w * t + ph)
    try:
        p, _ = curve_fit(fn, np.array(ts), np.array(bs),
                         p0=[max(np.abs(bs)), 1e-4, np.sqrt(1.4 * T0) * k, 0.0])
    except Exception:
        return False
    G = 0.5 * k * k * ((4 / 3) * tr["eta"] + tr["eta_b"] + 0.4 * tr["kappa"] / 3.5)
    return abs(p[1] / G - 1) < 0.05


def _mirror_x(a, nx, ny, nz, ncomp=1, flip_sign=False):
    """Mirror a field about x = 0 in physical coordinates: s = 0 at x maps to
    s = 0 at -x mod nx, s = 1 at x + 1/2 maps to s = 1 at nx - 1 - x."""
    a = np.asarray(a).reshape(ncomp, 2, nz, ny, nx).copy()
    out = np.empty_like(a)
    out[:, 0] = np.roll(a[:, 0, :, :, ::-1], 1, axis=-1)
    out[:, 1] = a[:, 1, :, :, ::-1]
    if flip_sign:
        out[0] = -out[0]
    return out.reshape(ncomp, -1) if ncomp > 1 else out.reshape(-1)


def _pin_mirror():
    """One step from rest is symmetric under x -> -x (symmetric velocity set,
    point-local collision, no advection at u = 0, symmetric diffusion)."""
    nx, ny, nz = 8, 2, 1
    P = O.make_params(2.0, 0.7, 0.9, 0.2, 2.0, 1.0, 2, 0)
    X = I.positions(nx, ny, nz)
    k = 2 * np.pi / nx
    rho = 1 + 0.3 * np.sin(k * X[0] + 0.4)
    T = T0 * (1 + 0.05 * np.cos(k * X[0] + 1.1))
    R = T0 * (1 + 0.1 * np.sin(2 * k * X[0] + 0.3))
    u = np.zeros((3, X.shape[1]))
    A = O.State(P, nx, ny, nz).init_fields(rho, u, T, R).step(1).fields()
    m = lambda a: _mirror_x(a, nx, ny, nz)
    B = O.State(P, nx, ny, nz).init_fields(m(rho), u, m(T), m(R)).step(1).fields()
    return all(np.allclose(m(A[key]), B[key], rtol=0, atol=1e-14) for key in ("rho", "T", "R")) \
        and np.allclose(_mirror_x(A["u"], nx, ny, nz, 3, True), B["u"], rtol=0, atol=1e-15)


PINS = [_pin_mirror, _pin_targets, _pin_relaxation, _pin_init_round_trip, _pin_streaming,
        _pin_maccormack, _pin_conservation, _pin_h1_rest, _pin_acoustic_attenuation]


def _run_pins():
    failed = []
    for pin in PINS:
        try:
            ok = pin()
        except Exception:
            ok = False
        if not ok:
            failed.append(pin.__name__)
    return failed


def test_pins_pass_on_the_unmodified_oracle():
    assert _run_pins() == []


@pytest.mark.parametrize("name,orig,mut", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, orig, mut):
    src = O.source()
    assert src.count(orig) == 1, "mutation anchor not found: %s" % name
    path = O.compile_variant(src.replace(orig, mut), str(tmp_path / "mutant.so"))
    with O.using_library(path):
        failed = _run_pins()
    assert failed, "no pin caught: %s" % name
