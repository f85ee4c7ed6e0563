"""Host-side parameter mapping of the reduced ES-BGK model, written from the
paper for the oracle (TEST INFRASTRUCTURE; the CUDA library has its own).

Sec. 3, eq. thetadef and the hydrodynamic paragraph of Sec. 4:
    gamma  = (5 + delta) / (3 + delta)
    eta    = p tau / (B - b),          B = 1 + tau / tau1     (eq. viscosities)
    eta_b  = 2 delta / (3 (3 + delta)) p tau1                 (eq. viscosities)
    kappa  = 5 p tau / (2 B) (1 + k_r)
    Pr     = (B / (B - b)) (1 + delta / 5) / (1 + k_r)
All at the reference state p0 = rho0 * theta0 of the lattice.
"""
import math

THETA0 = 0.2948964908710633  # Sec. 5, Table 1


def delta_from_gamma(gamma):
    """Invert gamma = (5 + delta)/(3 + delta) (Sec. 4, hydrodynamics)."""
    return (5.0 - 3.0 * gamma) / (gamma - 1.0)


def gamma_from_delta(delta):
    return (5.0 + delta) / (3.0 + delta)


def c_delta(delta):
    """eta_b / (p tau1) from eq. viscosities."""
    return 2.0 * delta / (3.0 * (3.0 + delta))


def relax_from_gas(gamma, eta, eta_B, kappa, b=0.0, rho0=1.0, theta0=THETA0):
    """(delta, tau, tau1, b, k_r) from (gamma, eta, eta_B, kappa, b).

    tau1 from eta_b = c_delta p0 tau1; tau from eta (B - b) = p0 tau with
    B = 1 + tau/tau1, i.e. tau = eta (1 - b) / (p0 - eta/tau1); k_r from
    kappa = kappa_T (1 + k_r), kappa_T = 5 p0 tau / (2 B).
    Raises ValueError where no positive (tau, tau1) or no k_r >= 0 exists.
    """
    delta = delta_from_gamma(gamma)
    if not delta >= 0.0:
        raise ValueError("gamma must lie in (1, 5/3]")
    p0 = rho0 * theta0
    if delta == 0.0:
        raise ValueError("delta = 0 (monoatomic) has no bulk viscosity to set tau1 from")
    tau1 = eta_B / (c_delta(delta) * p0)
    denom = p0 - eta / tau1
    tau = eta * (1.0 - b) / denom if denom != 0.0 else float("nan")
    if not (tau1 > 0.0 and tau > 0.0 and math.isfinite(tau)):
        raise ValueError("no positive tau for eta_B/eta = %g with b = %g" % (eta_B / eta, b))
    B = 1.0 + tau / tau1
    kappa_T = 5.0 * p0 * tau / (2.0 * B)
    kr = kappa / kappa_T - 1.0
    if kr < -1e-12:
        raise ValueError("kappa below kappa_T: k_r = %g < 0" % kr)
    return delta, tau, tau1, b, max(kr, 0.0)


def gas_from_nondim(gamma, nu, lam, Pr, rho0=1.0):
    """(eta, eta_B, kappa) from kinematic viscosity nu, bulk-to-shear ratio lam
    and Prandtl number Pr = eta c_p / kappa, c_p = (5 + delta)/2 per unit mass."""
    delta = delta_from_gamma(gamma)
    eta = rho0 * nu
    cp = (5.0 + delta) / 2.0
    return eta, lam * eta, eta * cp / Pr


def transport(delta, tau, tau1, b, kr, p=THETA0):
    """Closed-form transport coefficients of the model (Sec. 4)."""
    B = 1.0 + tau / tau1
    eta = p * tau / (B - b)
    eta_b = c_delta(delta) * p * tau1
    kappa_T = 5.0 * p * tau / (2.0 * B)
    kappa = kappa_T * (1.0 + kr)
    Pr = (B / (B - b)) * (1.0 + delta / 5.0) / (1.0 + kr)
    return {"eta": eta, "eta_b": eta_b, "kappa_T": kappa_T, "kappa": kappa, "Pr": Pr,
            "gamma": gamma_from_delta(delta)}


def nsub_for(delta, tau, tau1, kr, theta_max, ndim, dt=1.0):
    """FTCS sub-steps for the rotational diffusion: the scheme on
    theta_R = 2 E_R/(delta rho) has diffusivity D = 2 kappa_R/(delta rho)
    = 5 k_r tau theta / (delta B); explicit stability in ndim dimensions needs
    2 ndim D dt/nsub <= 1, kept at 0.9 of that with theta_max = 1.25 x the
    largest initial theta."""
    if kr <= 0.0 or ndim == 0:
        return 1
    B = 1.0 + tau / tau1
    D = 5.0 * kr * tau * (1.25 * theta_max) / (delta * B)
    return max(1, int(math.ceil(2.0 * ndim * D * dt / 0.9)))
