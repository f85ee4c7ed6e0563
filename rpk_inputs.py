"""Seeded synthetic inputs for the reduced polyatomic lattice-Boltzmann step.

This module is shared by the tests, the benchmark and the smoke check. It
generates hydrodynamic fields (rho, u, theta_T, theta_R) only; it holds none of
the method's arithmetic. Every generator takes the lattice reference
temperature ``theta0`` from its caller.

Field layout (the library's public layout): a scalar field is a float64 array of
2*nx*ny*nz entries indexed p = ((s*nz + z)*ny + y)*nx + x; sublattice s = 1 sits
at (x, y, z) + (1/2, 1/2, 1/2) in units of the sublattice spacing. ``u`` has
shape (3, npts).
"""
import numpy as np

SEED = 20220113


def positions(nx, ny, nz):
    """Physical coordinates (3, npts) of every BCC point in sublattice units."""
    s, z, y, x = np.meshgrid(np.arange(2), np.arange(nz), np.arange(ny), np.arange(nx),
                             indexing="ij")
    off = 0.5 * s
    return np.stack([(x + off).ravel(), (y + off).ravel(), (z + off).ravel()]).astype(np.float64)


def uniform(nx, ny, nz, theta0, rho=1.0, u=(0.0, 0.0, 0.0), T=None, R=None):
    n = 2 * nx * ny * nz
    T = theta0 if T is None else T
    R = T if R is None else R
    return {"rho": np.full(n, float(rho)), "u": np.tile(np.asarray(u, float)[:, None], (1, n)),
            "T": np.full(n, float(T)), "R": np.full(n, float(R))}


def shear_wave(nx, ny, nz, theta0, amp=1e-3, mode=1, axis=0, comp=1):
    """u_comp = amp sin(k x_axis), k = 2 pi mode / n_axis; rho = 1, theta = theta0."""
    X = positions(nx, ny, nz)
    L = (nx, ny, nz)[axis]
    k = 2.0 * np.pi * mode / L
    f = uniform(nx, ny, nz, theta0)
    f["u"][comp] = amp * np.sin(k * X[axis])
    return f, k


def acoustic_wave(nx, ny, nz, theta0, gamma, amp=1e-3, mode=1):
    """Standing adiabatic wave along x: rho = 1 + amp cos kx,
    theta = theta0 (1 + (gamma - 1) amp cos kx), u = 0, theta_R = theta_T."""
    X = positions(nx, ny, nz)
    k = 2.0 * np.pi * mode / nx
    cx = np.cos(k * X[0])
    f = uniform(nx, ny, nz, theta0)
    f["rho"] = 1.0 + amp * cx
    f["T"] = theta0 * (1.0 + (gamma - 1.0) * amp * cx)
    f["R"] = f["T"].copy()
    return f, k


def thermal_wave(nx, ny, nz, theta0, amp=1e-3, mode=1):
    """Isobaric entropy wave along x: theta = theta0 (1 + amp sin kx),
    rho = 1/(1 + amp sin kx), u = 0, theta_R = theta_T."""
    X = positions(nx, ny, nz)
    k = 2.0 * np.pi * mode / nx
    sx = np.sin(k * X[0])
    f = uniform(nx, ny, nz, theta0)
    f["T"] = theta0 * (1.0 + amp * sx)
    f["R"] = f["T"].copy()
    f["rho"] = 1.0 / (1.0 + amp * sx)
    return f, k


def fourier_modes(nx, ny, nz, theta0, nmodes=8, amp=1e-3, seed=SEED, nmax=3):
    """Uniform rho = 1, theta = theta0 plus ``nmodes`` seeded Fourier modes.

    Wave vectors n in [-nmax, nmax]^3 \\ {0}, distinct up to sign, restricted to
    axes with more than one cell (fewer modes when fewer exist; none on a box of
    one cell); each mode carries random-phase perturbations of amplitude ``amp``
    in rho, theta and in u (a random direction, so it has shear and
    longitudinal parts). Returns (fields, list of mode dicts).
    """
    rng = np.random.default_rng(seed)
    X = positions(nx, ny, nz)
    L = np.array([nx, ny, nz], float)
    f = uniform(nx, ny, nz, theta0)
    active = [d for d in range(3) if (nx, ny, nz)[d] > 1]
    # every admissible wave vector, one representative per +-pair
    cands = []
    rngs = [range(-nmax, nmax + 1) if d in active else range(1) for d in range(3)]
    for a in rngs[0]:
        for b in rngs[1]:
            for c in rngs[2]:
                n = (a, b, c)
                if any(n) and (-a, -b, -c) not in cands:
                    cands.append(n)
    count = min(nmodes, len(cands))
    picks = rng.permutation(len(cands))[:count]
    modes = []
    for idx in picks:
        n = np.array(cands[idx], int)
        k = 2.0 * np.pi * n / L
        ph = k @ X
        a = amp * rng.uniform(0.5, 1.0, size=3)
        phi = rng.uniform(0, 2 * np.pi, size=5)
        d = rng.normal(size=3)
        for dd in range(3):
            if dd not in active:
                d[dd] = 0.0
        nd = np.linalg.norm(d)
        d = d / nd if nd > 0 else d
        f["rho"] += a[0] * np.cos(ph + phi[0])
        f["T"] += theta0 * a[1] * np.cos(ph + phi[1])
        f["u"] += (a[2] * np.cos(ph + phi[2]))[None, :] * d[:, None]
        modes.append({"n": n, "k": k, "dir": d})
    f["R"] = f["T"].copy()
    return f, modes


def shock_tube(nx, theta0, rho_l=1.0, p_l=1.0, rho_r=0.125, p_r=0.1, ny=1, nz=1):
    """Quasi-1-D Riemann problem along x, diaphragm at x = nx/2 (points whose
    physical x < nx/2 take the left state). Physical pressure p maps to lattice
    temperature theta = theta0 p/rho (theta_phys = 1 -> theta0); u = 0 and
    theta_R = theta_T. Returns (fields, reservoir states (12,)): rho, ux, uy, uz,
    T, R of the low-x then the high-x state."""
    X = positions(nx, ny, nz)
    left = X[0] < 0.5 * nx
    f = uniform(nx, ny, nz, theta0)
    T_l, T_r = theta0 * p_l / rho_l, theta0 * p_r / rho_r
    f["rho"] = np.where(left, rho_l, rho_r)
    f["T"] = np.where(left, T_l, T_r)
    f["R"] = f["T"].copy()
    res = np.array([rho_l, 0, 0, 0, T_l, T_l, rho_r, 0, 0, 0, T_r, T_r], float)
    return f, res


def taylor_green(n, theta0, u0, rho0=1.0):
    """3-D Taylor-Green vortex on an n^3 periodic box, wavelength n:
    u = u0 (sin kx cos ky cos kz, -cos kx sin ky cos kz, 0),
    p = p0 + rho0 u0^2/16 (cos 2kx + cos 2ky)(cos 2kz + 2), theta = theta0,
    rho = p / theta0 (isothermal start), theta_R = theta_T."""
    X = positions(n, n, n)
    k = 2.0 * np.pi / n
    x, y, z = X
    f = uniform(n, n, n, theta0)
    f["u"][0] = u0 * np.sin(k * x) * np.cos(k * y) * np.cos(k * z)
    f["u"][1] = -u0 * np.cos(k * x) * np.sin(k * y) * np.cos(k * z)
    p = rho0 * theta0 + rho0 * u0 ** 2 / 16.0 * (np.cos(2 * k * x) + np.cos(2 * k * y)) * (
        np.cos(2 * k * z) + 2.0)
    f["rho"] = p / theta0
    return f


def random_smooth(nx, ny, nz, theta0, seed=SEED, amp=0.02, aniso_R=0.02):
    """Smooth but generic state: a few random modes of amplitude ``amp`` in
    rho, u and theta, plus theta_R != theta_T (relative offset ``aniso_R``)."""
    f, _ = fourier_modes(nx, ny, nz, theta0, nmodes=4, amp=amp, seed=seed, nmax=2)
    rng = np.random.default_rng(seed + 1)
    X = positions(nx, ny, nz)
    k = 2.0 * np.pi / np.array([nx, ny, nz], float)
    ph = rng.uniform(0, 2 * np.pi, 3)
    f["R"] = f["T"] * (1.0 + aniso_R * np.cos(k[0] * X[0] + ph[0]) * np.cos(k[1] * X[1] + ph[1]))
    return f


def tile(fields, nx, ny, nz, reps):
    """Repeat a periodic field set on an (nx, ny, nz) box reps = (rx, ry, rz)
    times along each axis; the result lives on (rx nx, ry ny, rz nz)."""
    rx, ry, rz = reps

    def t(a, ncomp):
        a = np.asarray(a).reshape(ncomp, 2, nz, ny, nx)
        return np.tile(a, (1, 1, rz, ry, rx)).reshape(ncomp, -1)

    return {"rho": t(fields["rho"], 1)[0], "u": t(fields["u"], 3),
            "T": t(fields["T"], 1)[0], "R": t(fields["R"], 1)[0]}


def tube_sweep(ntubes, theta0, gamma=1.4, seed=SEED, L=(500, 4000), ratio=(2.0, 20.0),
               kn=(1e-3, 1e-1), lam=(0.3, 2.0), pr=0.71, run_fraction=0.35):
    """Seeded batch of quasi-1-D Riemann problems (the batched shock-tube
    sweep): per tube a length nx ~ U[L], pressure ratio ~ U[ratio] with the
    right state on the left state's isentrope (rho_R = ratio^(-1/gamma), left
    rho = 1, p = 1), Knudsen number log-uniform in ``kn``, eta_B/eta ~ U[lam],
    Prandtl number ``pr``, and a run of round(run_fraction * nx / c_s) steps
    (c_s = sqrt(gamma theta0)). Returns (specs, fields) where specs is a list of
    dicts (nx, nsteps, ratio, kn, lam, pr, res) and fields the concatenated
    initial fields (tube after tube, 2 nx points each)."""
    rng = np.random.default_rng(seed)
    cs = np.sqrt(gamma * theta0)
    specs, parts = [], []
    for _ in range(ntubes):
        nx = int(rng.integers(L[0], L[1] + 1))
        r = float(rng.uniform(*ratio))
        k = float(np.exp(rng.uniform(np.log(kn[0]), np.log(kn[1]))))
        la = float(rng.uniform(*lam))
        f, res = shock_tube(nx, theta0, rho_r=r ** (-1.0 / gamma), p_r=1.0 / r)
        specs.append({"nx": nx, "nsteps": int(round(run_fraction * nx / cs)), "ratio": r,
                      "kn": k, "lam": la, "pr": pr, "res": res})
        parts.append(f)
    fields = {"rho": np.concatenate([p["rho"] for p in parts]),
              "u": np.concatenate([p["u"] for p in parts], axis=1),
              "T": np.concatenate([p["T"] for p in parts]),
              "R": np.concatenate([p["R"] for p in parts])}
    return specs, fields
