/*
 * rpk_oracle.c -- plain FP64 CPU oracle for one lattice-Boltzmann time step of
 * the reduced polyatomic ES-BGK model of Kolluru, Atif & Ansumali,
 * "Reduced kinetic model of polyatomic gases" (arXiv 2201.05280).
 *
 * TEST INFRASTRUCTURE. This file exists to check the CUDA library, not to be
 * used by it: only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load it. It shares no code, header or table with the CUDA path.
 *
 * Everything is double precision, single threaded, written as plain loops in
 * the order the paper states the scheme, so that each function can be read
 * against the paper:
 *
 *   lattice          Sec. 5, Table 1 (RD3Q41 velocities and weights, theta0)
 *   bcc layout       Sec. 5 (two simple-cubic sublattices offset by half a
 *                    spacing in every direction)
 *   discrete targets f^ES and f^Eq are not written out by the paper; this
 *                    oracle uses the third-order Hermite expansion about the
 *                    Table 1 weights of a Gaussian with mean u and covariance
 *                    Lambda (Sec. 2, eq. lambdaij, for the covariance)
 *   collision        Sec. 5, eq. discrete_f1 and the collision term below it
 *   g-transform      Sec. 5, trapezoid rule: g = f - (dt/2) Omega, the explicit
 *                    update for g and the g/f moment relations
 *   rotational part  Sec. 4, eq. kinEqBGK (second line) and
 *                    eq. rotHeatFlux_simple; solved here in conservative flux
 *                    form with the same trapezoid rule for its relaxation
 *                    (the paper leaves the solver free, end of Sec. 5)
 *   diagnostics      Sec. 4 (conservation laws, eq. ConservedMomEq; H1 of the
 *                    H-theorem paragraph with k = -delta/2)
 *   diffuse walls    Sec. 6 (the diffusive wall the paper cites for its Couette
 *                    and cavity flows; the reading is stated at wall_density)
 *
 * Grid layout shared with the library's public interface: a scalar field has
 * 2*nx*ny*nz entries indexed p = ((s*nz + z)*ny + y)*nx + x, s = 0 for the
 * corner sublattice and s = 1 for the body-centre one (physical position
 * (x, y, z) + s*(1/2, 1/2, 1/2) in units of the sublattice spacing). Vector
 * fields store their three components as three such planes. Populations are
 * stored point-major here: g[p*41 + i].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define Q 41

/* Sec. 5, Table 1: reference temperature of the RD3Q41 lattice. */
static const double THETA0 = 0.2948964908710633;

static double C[Q][3]; /* velocities in units of the sublattice spacing */
static double W[Q];    /* weights */
static double H2[Q][3][3];    /* Hermite tensors about theta0, see ora_target */
static double H3[Q][3][3][3];
static int lattice_built = 0;

static double kron(int a, int b) { return a == b ? 1.0 : 0.0; }

typedef struct {
    double delta; /* rotational degrees of freedom (Sec. 3, eq. thetadef) */
    double tau;   /* ES-BGK relaxation time (Sec. 4, eq. kinEqBGK) */
    double tau1;  /* BGK relaxation time to theta (Sec. 4, eq. kinEqBGK) */
    double b;     /* ES-BGK parameter (Sec. 2, eq. lambdaij) */
    double kr;    /* kappa_R / kappa_T (Sec. 4, conductivity paragraph) */
    double dt;    /* time step (1 in lattice units) */
    int nsub;     /* FTCS sub-steps of the rotational diffusion per time step */
    int bcx;      /* 0: periodic in x; 1: fixed reservoirs beyond both x ends; 2: diffuse
                     walls normal to x (xwall) */
    int diff;     /* rotational diffusion: 0 FTCS sub-steps (Sec. 5); 1 one backward-Euler
                     step (variant for quasi-1-D tubes: ny = nz = 1, bcx = 1) */
    int rot_mode; /* 0: conservative form, the state holds Er (auxiliary energy density);
                     1: the paper's theta_R solver (Sec. 5, four steps), the state holds theta_R */
    int bcy;      /* 0: periodic in y; 1: diffuse walls normal to y (Sec. 6, startup and
                     thermal Couette flows), see wall_fluxes below */
    double wall[8]; /* bcy = 1: ux, uy, uz, theta of the low-y wall, then of the high-y wall */
    double xwall[8]; /* bcx = 2: ux, uy, uz, theta of the low-x wall, then of the high-x wall */
} ora_params;

static void put(int i, double cx, double cy, double cz, double w)
{
    C[i][0] = cx; C[i][1] = cy; C[i][2] = cz; W[i] = w;
}

/* Sec. 5, Table 1: the 41 velocities in six shells and their weights. */
static void build_lattice(void)
{
    const double t = THETA0;
    const double w_rest = (52.0 - 323.0 * t + 921.0 * t * t - 1036.0 * t * t * t) / 52.0;
    const double w_100 = t * (12.0 - 38.0 * t + 63.0 * t * t) / 39.0;
    const double w_200 = t * (3.0 - 29.0 * t + 84.0 * t * t) / 312.0;
    const double w_110 = t * (45.0 * t - 6.0 - 77.0 * t * t) / 26.0;
    const double w_111 = t * (20.0 - 163.0 * t + 378.0 * t * t) / 312.0;
    const double w_hhh = 8.0 * t * (4.0 - 17.0 * t + 21.0 * t * t) / 39.0;
    int n = 0, a, b, sa, sb, sc;
    double v[3];

    put(n++, 0.0, 0.0, 0.0, w_rest);
    for (a = 0; a < 3; a++)
        for (sa = -1; sa <= 1; sa += 2) {
            v[0] = v[1] = v[2] = 0.0; v[a] = sa;
            put(n++, v[0], v[1], v[2], w_100);
        }
    for (a = 0; a < 3; a++)
        for (sa = -1; sa <= 1; sa += 2) {
            v[0] = v[1] = v[2] = 0.0; v[a] = 2.0 * sa;
            put(n++, v[0], v[1], v[2], w_200);
        }
    for (a = 0; a < 3; a++)
        for (b = a + 1; b < 3; b++)
            for (sa = -1; sa <= 1; sa += 2)
                for (sb = -1; sb <= 1; sb += 2) {
                    v[0] = v[1] = v[2] = 0.0; v[a] = sa; v[b] = sb;
                    put(n++, v[0], v[1], v[2], w_110);
                }
    for (sa = -1; sa <= 1; sa += 2)
        for (sb = -1; sb <= 1; sb += 2)
            for (sc = -1; sc <= 1; sc += 2)
                put(n++, sa, sb, sc, w_111);
    for (sa = -1; sa <= 1; sa += 2)
        for (sb = -1; sb <= 1; sb += 2)
            for (sc = -1; sc <= 1; sc += 2)
                put(n++, 0.5 * sa, 0.5 * sb, 0.5 * sc, w_hhh);
    /* Hermite tensors of each velocity about the lattice temperature t:
     * H2_ab = c_a c_b - t d_ab, H3_abc = c_a c_b c_c - t (d_ab c_c + d_bc c_a + d_ca c_b) */
    for (n = 0; n < Q; n++) {
        const double *v = C[n];
        int c;
        for (a = 0; a < 3; a++)
            for (b = 0; b < 3; b++) {
                H2[n][a][b] = v[a] * v[b] - t * kron(a, b);
                for (c = 0; c < 3; c++)
                    H3[n][a][b][c] = v[a] * v[b] * v[c] -
                                     t * (kron(a, b) * v[c] + kron(b, c) * v[a] + kron(c, a) * v[b]);
            }
    }
    lattice_built = 1;
}

static void need_lattice(void)
{
    if (!lattice_built) build_lattice();
}

double ora_theta0(void) { return THETA0; }

void ora_lattice(double *c, double *w)
{
    int i, a;
    need_lattice();
    for (i = 0; i < Q; i++) {
        for (a = 0; a < 3; a++) c[3 * i + a] = C[i][a];
        w[i] = W[i];
    }
}

/*
 * Discrete anisotropic Gaussian: third-order Hermite expansion about the
 * lattice weights of a Gaussian with density rho, mean u and covariance Lam:
 *   f_i = w_i [ rho + rho u.c/t0 + A2:H2(c)/(2 t0^2) + A3:H3(c)/(6 t0^3) ]
 *   A2_ab  = rho (u_a u_b + D_ab),  D = Lam - t0 I
 *   A3_abc = rho (u_a u_b u_c + D_ab u_c + D_bc u_a + D_ca u_b)
 *   H2_ab  = c_a c_b - t0 d_ab
 *   H3_abc = c_a c_b c_c - t0 (d_ab c_c + d_bc c_a + d_ca c_b)
 * With Lam = theta I this is the discrete Maxwellian f^Eq(rho, u, theta) of
 * the BGK term; with Lam = theta_T I + b sigma / rho it is the discrete
 * ES target (Sec. 2, eq. lambdaij; Sec. 5 collision term).
 */
void ora_target(double rho, const double *u, const double *Lam, double *f)
{
    const double t0 = THETA0;
    double D[3][3], A2[3][3], A3[3][3][3];
    int i, a, b, c;
    need_lattice();
    for (a = 0; a < 3; a++)
        for (b = 0; b < 3; b++)
            D[a][b] = Lam[3 * a + b] - t0 * kron(a, b);
    for (a = 0; a < 3; a++)
        for (b = 0; b < 3; b++)
            A2[a][b] = rho * (u[a] * u[b] + D[a][b]);
    for (a = 0; a < 3; a++)
        for (b = 0; b < 3; b++)
            for (c = 0; c < 3; c++)
                A3[a][b][c] = rho * (u[a] * u[b] * u[c] + D[a][b] * u[c] +
                                     D[b][c] * u[a] + D[c][a] * u[b]);
    for (i = 0; i < Q; i++) {
        const double *v = C[i];
        double h1 = 0.0, h2 = 0.0, h3 = 0.0;
        for (a = 0; a < 3; a++) h1 += rho * u[a] * v[a];
        for (a = 0; a < 3; a++)
            for (b = 0; b < 3; b++)
                h2 += A2[a][b] * H2[i][a][b];
        for (a = 0; a < 3; a++)
            for (b = 0; b < 3; b++)
                for (c = 0; c < 3; c++)
                    h3 += A3[a][b][c] * H3[i][a][b][c];
        f[i] = W[i] * (rho + h1 / t0 + h2 / (2.0 * t0 * t0) + h3 / (6.0 * t0 * t0 * t0));
    }
}

/* Derived relaxation constants of Sec. 5: 1/tau* = 1/tau + 1/tau1 and
 * beta* = dt / (2 tau* + dt). */
static double tau_star(const ora_params *P) { return 1.0 / (1.0 / P->tau + 1.0 / P->tau1); }
static double beta_star(const ora_params *P) { return P->dt / (2.0 * tau_star(P) + P->dt); }

typedef struct {
    double rho, u[3];
    double thetaTg;     /* translational temperature of g */
    double T, R;        /* theta_T(f) and theta_R of the f-level state */
    double theta;       /* eq. thetadef: (3 T + delta R) / (3 + delta) */
    double sigma[3][3]; /* stress of f, a density: P - rho u u - rho T I */
} moments;

/*
 * Moments of the f-level state from the stored auxiliary population g and the
 * stored auxiliary rotational energy Er.
 *   rho, u: Sec. 5, equal for g and f.
 *   theta_T(g) = theta_T(f) + a (theta_T(f) - theta_R),
 *       a = delta dt / (2 tau1 (3 + delta))          (Sec. 5, g/f relations)
 *   Er = E_R - (dt/2) (delta rho / 2)(theta - theta_R)/tau1, the same
 *       trapezoid transform applied to the relaxation in eq. kinEqBGK; with
 *       eq. thetadef, theta - theta_R = 3 (T - R)/(3 + delta), so
 *       Rt := 2 Er/(delta rho) = R - X (T - R),  X = 3 dt / (2 tau1 (3+delta))
 *       (X is the constant of the paper's rotational half-step, Sec. 5).
 *   The two relations form a 2x2 linear system for (T, R), solved by Cramer.
 *   sigma(g) = sigma(f) (1 + dt/(2 tau*) - b dt/(2 tau))   (Sec. 5).
 */
static void recover(const ora_params *P, const double *g, double Er, moments *m)
{
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0}, Pt[3][3];
    double u2 = 0.0, trP = 0.0, a_, X, det, Rt, fac;
    int i, a, b;
    need_lattice();
    for (a = 0; a < 3; a++)
        for (b = 0; b < 3; b++) Pt[a][b] = 0.0;
    for (i = 0; i < Q; i++) {
        rho += g[i];
        for (a = 0; a < 3; a++) j[a] += g[i] * C[i][a];
        for (a = 0; a < 3; a++)
            for (b = 0; b < 3; b++) Pt[a][b] += g[i] * C[i][a] * C[i][b];
    }
    m->rho = rho;
    for (a = 0; a < 3; a++) m->u[a] = j[a] / rho;
    for (a = 0; a < 3; a++) u2 += m->u[a] * m->u[a];
    for (a = 0; a < 3; a++) trP += Pt[a][a];
    /* Sec. 5: theta_T = (sum g c^2 - rho u^2) / (3 rho) */
    m->thetaTg = (trP - rho * u2) / (3.0 * rho);

    a_ = P->delta * P->dt / (2.0 * P->tau1 * (3.0 + P->delta));
    X = 3.0 * P->dt / (2.0 * P->tau1 * (3.0 + P->delta));
    if (P->rot_mode == 1) {
        /* paper mode: the state is theta_R itself; the g-level translational
         * temperature relation (1 + a) T - a R = thetaTg gives T */
        m->R = Er;
        m->T = (m->thetaTg + a_ * m->R) / (1.0 + a_);
    } else {
        Rt = 2.0 * Er / (P->delta * rho);
        /* (1 + a) T - a R = thetaTg ;  -X T + (1 + X) R = Rt */
        det = (1.0 + a_) * (1.0 + X) - a_ * X;
        m->T = (m->thetaTg * (1.0 + X) + a_ * Rt) / det;
        m->R = ((1.0 + a_) * Rt + X * m->thetaTg) / det;
    }
    m->theta = (3.0 * m->T + P->delta * m->R) / (3.0 + P->delta);

    fac = 1.0 + P->dt / (2.0 * tau_star(P)) - P->b * P->dt / (2.0 * P->tau);
    for (a = 0; a < 3; a++)
        for (b = 0; b < 3; b++)
            m->sigma[a][b] = (Pt[a][b] - rho * m->u[a] * m->u[b] -
                              rho * m->thetaTg * kron(a, b)) / fac;
}

/* The two discrete targets of the collision term (Sec. 5):
 * f^ES(rho, u, T I + b sigma/rho) and f^Eq(rho, u, theta I). */
static void targets(const ora_params *P, const moments *m, double *fES, double *fEq)
{
    double LamES[9], LamEq[9];
    int a, b;
    for (a = 0; a < 3; a++)
        for (b = 0; b < 3; b++) {
            LamES[3 * a + b] = m->T * kron(a, b) + P->b * m->sigma[a][b] / m->rho;
            LamEq[3 * a + b] = m->theta * kron(a, b);
        }
    ora_target(m->rho, m->u, LamES, fES);
    ora_target(m->rho, m->u, LamEq, fEq);
}

/* One collision at one point, in place (no streaming):
 *   g' = (1 - 2 beta*) g + 2 beta* tau* (f^ES/tau + f^Eq/tau1)       (Sec. 5)
 *   Er' = Er + dt (delta rho / 2)(theta - theta_R)/tau1
 * The second line is the trapezoid rule for the rotational relaxation in
 * eq. kinEqBGK written for the transformed Er; it carries exactly the energy
 * that the first line moves out of (or into) sum g c^2/2. */
static void collide(const ora_params *P, double *g, double *Er, moments *m_out)
{
    moments m;
    double fES[Q], fEq[Q];
    const double ts = tau_star(P), bs = beta_star(P);
    int i;
    recover(P, g, *Er, &m);
    targets(P, &m, fES, fEq);
    for (i = 0; i < Q; i++)
        g[i] = (1.0 - 2.0 * bs) * g[i] + 2.0 * bs * ts * (fES[i] / P->tau + fEq[i] / P->tau1);
    if (P->rot_mode != 1) /* paper mode relaxes theta_R in the transport stage */
        *Er = *Er + P->dt * (P->delta * m.rho / 2.0) * (m.theta - m.R) / P->tau1;
    if (m_out) *m_out = m;
}

/* f from g: g = f - (dt/2)(f^mix - f)/tau*, f^mix = tau*(f^ES/tau + f^Eq/tau1),
 * hence f = (2 tau* g + dt f^mix) / (2 tau* + dt). */
static void f_from_g(const ora_params *P, const double *g, double Er, double *f, moments *m)
{
    double fES[Q], fEq[Q];
    const double ts = tau_star(P);
    int i;
    recover(P, g, Er, m);
    targets(P, m, fES, fEq);
    for (i = 0; i < Q; i++) {
        double fmix = ts * (fES[i] / P->tau + fEq[i] / P->tau1);
        f[i] = (2.0 * ts * g[i] + P->dt * fmix) / (2.0 * ts + P->dt);
    }
}

/*
 * Initial state from hydrodynamic fields: f = f^Eq(rho, u, T I) (isotropic,
 * sigma = 0, so f^ES = f and only the BGK term of Omega is non-zero), then
 *   g  = f - (dt/2) Omega(f)
 *   Er = E_R - (dt/2)(delta rho/2)(theta - R)/tau1,  E_R = delta rho R / 2.
 */
void ora_point_init(const ora_params *P, double rho, const double *u, double T, double R,
                    double *g, double *Er)
{
    double LamT[9], LamTh[9], f[Q], fEq[Q];
    const double theta = (3.0 * T + P->delta * R) / (3.0 + P->delta);
    int a, b, i;
    for (a = 0; a < 3; a++)
        for (b = 0; b < 3; b++) {
            LamT[3 * a + b] = T * kron(a, b);
            LamTh[3 * a + b] = theta * kron(a, b);
        }
    ora_target(rho, u, LamT, f);
    ora_target(rho, u, LamTh, fEq);
    for (i = 0; i < Q; i++) {
        double Omega = (f[i] - f[i]) / P->tau + (fEq[i] - f[i]) / P->tau1;
        g[i] = f[i] - 0.5 * P->dt * Omega;
    }
    if (P->rot_mode == 1)
        *Er = R; /* paper mode: the state is theta_R */
    else
        *Er = 0.5 * P->delta * rho * R -
              0.5 * P->dt * (0.5 * P->delta * rho) * (theta - R) / P->tau1;
}

/* out: rho, ux, uy, uz, T, R, theta, thetaTg, sigma[9] (17 values) */
void ora_point_moments(const ora_params *P, const double *g, double Er, double *out)
{
    moments m;
    int a, b;
    recover(P, g, Er, &m);
    out[0] = m.rho;
    for (a = 0; a < 3; a++) out[1 + a] = m.u[a];
    out[4] = m.T; out[5] = m.R; out[6] = m.theta; out[7] = m.thetaTg;
    for (a = 0; a < 3; a++)
        for (b = 0; b < 3; b++) out[8 + 3 * a + b] = m.sigma[a][b];
}

void ora_point_collide(const ora_params *P, double *g, double *Er)
{
    collide(P, g, Er, NULL);
}

void ora_point_f(const ora_params *P, const double *g, double Er, double *f)
{
    moments m;
    f_from_g(P, g, Er, f, &m);
}

/* ------------------------------------------------------------------------ */
/* Grid: BCC layout, pull streaming and the rotational transport.           */

typedef struct {
    int nx, ny, nz;
    long n3;   /* nx*ny*nz */
    long npts; /* 2*n3 */
} grid;

static grid make_grid(int nx, int ny, int nz)
{
    grid G;
    G.nx = nx; G.ny = ny; G.nz = nz;
    G.n3 = (long)nx * ny * nz;
    G.npts = 2 * G.n3;
    return G;
}

static long pidx(const grid *G, int s, int x, int y, int z)
{
    return (((long)s * G->nz + z) * G->ny + y) * G->nx + x;
}

static int wrap(int a, int n) { a %= n; return a < 0 ? a + n : a; }

static int floor_div2(int a) { return (a >= 0) ? a / 2 : -((1 - a) / 2); }

/*
 * Source of the pull for population i at point (s, x, y, z): the particle that
 * arrives with velocity c_i left the position r - c_i one step earlier. In
 * half-spacing units the position is 2*idx + s on every axis; the source
 * sublattice s' is the parity of 2*idx + s - 2c (the same on all axes, since a
 * velocity is either all-integer or all-half-integer) and its index is
 * (2*idx + s - 2c - s')/2. Returns the point index, or -1 / -2 when the source
 * lies beyond the low / high x end (only with bcx = 1), -3 / -4 when it lies
 * beyond the low / high y wall (bcy = 1; also when it lies beyond an x wall as
 * well), -5 / -6 beyond the low / high x wall (bcx = 2).
 */
static long pull_source(const ora_params *P, const grid *G, int s, int x, int y, int z, int i)
{
    int idx[3] = {x, y, z}, n[3] = {G->nx, G->ny, G->nz}, src[3], sp, a;
    sp = (2 * idx[0] + s - (int)lround(2.0 * C[i][0])) & 1;
    for (a = 0; a < 3; a++) {
        int pos2 = 2 * idx[a] + s - (int)lround(2.0 * C[i][a]);
        src[a] = floor_div2(pos2 - sp);
    }
    if (P->bcy == 1) { /* checked first: a y wall emits what comes from beyond it and an x wall */
        if (src[1] < 0) return -3;
        if (src[1] >= n[1]) return -4;
    }
    if (P->bcx == 1) {
        if (src[0] < 0) return -1;
        if (src[0] >= n[0]) return -2;
    } else if (P->bcx == 2) {
        if (src[0] < 0) return -5;
        if (src[0] >= n[0]) return -6;
    } else {
        src[0] = wrap(src[0], n[0]);
    }
    src[1] = wrap(src[1], n[1]);
    src[2] = wrap(src[2], n[2]);
    return pidx(G, sp, src[0], src[1], src[2]);
}

/* Axis neighbour on the same sublattice: d = +1 or -1 along axis a. Returns -1
 * / -2 for a reservoir ghost beyond the low / high x end (bcx = 1 only),
 * -3 / -4 for the low / high y wall (bcy = 1 only) and -5 / -6 for the low /
 * high x wall (bcx = 2 only). */
static long axis_nb(const ora_params *P, const grid *G, long p, int a, int d)
{
    int x = (int)(p % G->nx);
    int y = (int)((p / G->nx) % G->ny);
    int z = (int)((p / ((long)G->nx * G->ny)) % G->nz);
    int s = (int)(p / G->n3);
    int idx[3] = {x, y, z}, n[3] = {G->nx, G->ny, G->nz};
    idx[a] += d;
    if (a == 0 && P->bcx == 1) {
        if (idx[0] < 0) return -1;
        if (idx[0] >= n[0]) return -2;
    }
    if (a == 0 && P->bcx == 2) {
        if (idx[0] < 0) return -5;
        if (idx[0] >= n[0]) return -6;
    }
    if (a == 1 && P->bcy == 1) {
        if (idx[1] < 0) return -3;
        if (idx[1] >= n[1]) return -4;
    }
    idx[a] = wrap(idx[a], n[a]);
    return pidx(G, s, idx[0], idx[1], idx[2]);
}

/* Reservoir ghost state (bcx = 1): one uniform equilibrium per x end. */
typedef struct {
    double g[Q], Er, rho, u[3], kap;
} ghost;

static double kappa_R(const ora_params *P, double rho, double theta)
{
    /* Sec. 4: kappa_T = 5 p tau / (2 B), B = 1 + tau/tau1, kappa_R = k_r kappa_T,
     * with p = rho theta. */
    const double B = 1.0 + P->tau / P->tau1;
    return P->kr * 5.0 * rho * theta * P->tau / (2.0 * B);
}

static void make_ghost(const ora_params *P, const double *st, ghost *gh)
{
    /* st: rho, ux, uy, uz, T, R */
    double theta = (3.0 * st[4] + P->delta * st[5]) / (3.0 + P->delta);
    ora_point_init(P, st[0], st + 1, st[4], st[5], gh->g, &gh->Er); /* theta_R in paper mode */
    gh->rho = st[0];
    gh->u[0] = st[1]; gh->u[1] = st[2]; gh->u[2] = st[3];
    gh->kap = kappa_R(P, st[0], theta);
}

/*
 * Diffuse walls (bcy = 1). The paper runs its Couette and cavity flows (Sec. 6)
 * with the diffusive wall of Ansumali & Karlin (2002), which it cites but does
 * not write out; this is that boundary condition in the following reading.
 * The walls are planes normal to y half way between layers of points: at
 * y = -1/4 and at y = ny - 1/4 in sublattice-spacing units (the layers sit at
 * y + s/2). A population whose pull source lies beyond a wall is not taken
 * from the lattice: the wall emits it as rho_w f^eq_i(1, u_w, theta_w), the
 * discrete Gaussian of the wall's velocity and temperature (full
 * accommodation), with rho_w set per (x, z) column so that the wall emits
 * into the column exactly the mass that left the column through it in the
 * same step:
 *   rho_w = (sum of the column's post-collision populations whose destination
 *            lies beyond the wall)
 *         / (sum of f^eq_i(1, u_w, theta_w) over the column's entries that
 *            the wall emits).
 * Mass is conserved exactly; momentum and energy are exchanged with the wall.
 * Walls normal to x (bcx = 2, for the square cavity of Sec. 6) are the same
 * with the axes exchanged, at x = -1/4 and x = nx - 1/4; where a population
 * crosses an x wall and a y wall (the corners) the y wall owns it.
 * The rotational energy sees the walls as Dirichlet boundaries at
 * theta_R = theta_w (the internal energy is accommodated as well): the
 * diffusive flux through the wall face of point p is
 * kappa_R(p) (theta_w - theta_R(p)) / d, d the distance from p to the wall
 * (1/4 or 3/4), and the advective flux through a wall is zero (the walls slide
 * tangentially: uy = 0). In the paper's theta_R mode the same Dirichlet value
 * enters through wall_ghost in the advection differences and the Laplacian.
 */

/* Index along axis a (not wrapped) of the destination of population i leaving
 * a point on sublattice s with index idx on that axis; the destination
 * sublattice is the parity of s + 2c, the same on all axes. */
static int dest_index(int s, int idx, int i, int a)
{
    const int c2 = (int)lround(2.0 * C[i][a]);
    const int sd = (s + c2) & 1;
    return floor_div2(2 * idx + s + c2 - sd);
}

/* Distance from point p (sublattice s) to the low (w = 0) or high (w = 1) y
 * wall when p is in the layer next to that wall. */
static double wall_distance(int s, int w)
{
    return w == 0 ? (2.0 * s + 1.0) / 4.0 : (3.0 - 2.0 * s) / 4.0;
}

/* Walls w = 0, 1 (low, high y) own the columns (x, z), walls w = 2, 3 (low,
 * high x) the columns (y, z); wall_slot gives the index of wall w's column
 * holding the point (x, y, z) in the arrays of wall_density. */
static long wall_slot(const grid *G, int w, int x, int y, int z)
{
    const long ny_cols = (long)G->nx * G->nz, nx_cols = (long)G->ny * G->nz;
    if (w < 2) return w * ny_cols + (long)z * G->nx + x;
    return 2 * ny_cols + (w - 2) * nx_cols + (long)z * G->ny + y;
}

/* Paper mode: theta_R on the axis neighbour beyond the wall of code q (<= -3)
 * of point p, given theta_R(p) = thp: the straight line through theta_w at the
 * wall (distance d from p), so that differences across the wall face see the
 * Dirichlet value theta_R = theta_w as the conservative form's flux does. */
static double wall_ghost(const ora_params *P, const grid *G, long p, long q, double thp)
{
    const int w = (int)(-3 - q), side = w & 1, s = (int)(p / G->n3);
    const double *wl = (w < 2) ? P->wall : P->xwall;
    const double d = wall_distance(s, side), thw = wl[4 * side + 3];
    return thw + (thw - thp) * (1.0 - d) / d;
}

/* rw[wall_slot(w, ...)]: rho_w of wall w for each of its columns, from the
 * post-collision populations gs; gw[w] is f^eq(1, u_w, theta_w). A population
 * whose destination (source) lies beyond a y wall belongs to that y wall even
 * if it lies beyond an x wall as well (the corners); the x walls take the
 * rest. */
static int wall_density(const ora_params *P, const grid *G, const double *gs, double gw[4][Q],
                        double *rw)
{
    const long nslot = 2 * (long)G->nx * G->nz + 2 * (long)G->ny * G->nz;
    double *out = (double *)calloc(nslot, sizeof(double));
    double *in = (double *)calloc(nslot, sizeof(double));
    long p, k;
    int i;
    if (!out || !in) {
        free(out); free(in);
        return 1;
    }
    for (p = 0; p < G->npts; p++) {
        const int x = (int)(p % G->nx), y = (int)((p / G->nx) % G->ny);
        const int z = (int)((p / ((long)G->nx * G->ny)) % G->nz), s = (int)(p / G->n3);
        for (i = 0; i < Q; i++) {
            const int yd = dest_index(s, y, i, 1), xd = dest_index(s, x, i, 0);
            const long q = pull_source(P, G, s, x, y, z, i);
            int wo = -1;
            if (P->bcy == 1 && yd < 0) wo = 0;
            else if (P->bcy == 1 && yd >= G->ny) wo = 1;
            else if (P->bcx == 2 && xd < 0) wo = 2;
            else if (P->bcx == 2 && xd >= G->nx) wo = 3;
            if (wo >= 0) out[wall_slot(G, wo, x, y, z)] += gs[p * Q + i];
            if (q <= -3) in[wall_slot(G, (int)(-3 - q), x, y, z)] += gw[-3 - q][i];
        }
    }
    for (k = 0; k < nslot; k++) rw[k] = (in[k] > 0.0) ? out[k] / in[k] : 0.0;
    free(out); free(in);
    return 0;
}

int ora_init(const ora_params *P, int nx, int ny, int nz, const double *rho, const double *u,
             const double *T, const double *R, double *g, double *Er)
{
    grid G = make_grid(nx, ny, nz);
    long p;
    need_lattice();
    for (p = 0; p < G.npts; p++) {
        double up[3] = {u[p], u[G.npts + p], u[2 * G.npts + p]};
        ora_point_init(P, rho[p], up, T[p], R[p], g + p * Q, Er + p);
    }
    return 0;
}

/*
 * Backward-Euler variant of the diffusion stage on one line of n points with
 * reservoir ends (the variant for quasi-1-D tubes): the flux-form equation
 * dEr/dt = d/dx(kappa_R d theta_R/dx), theta_R = 2 Er/(delta rho), taken in one
 * implicit step of dt with the face coefficients of the explicit scheme:
 *   (delta rho_p / 2) th_p - dt [K+ (th_{p+1} - th_p) - K- (th_p - th_{p-1})] = Er_p,
 *   K+- = (kap_p + kap_{p+-1}) / 2,
 * where th_{-1} = thl, kap_{-1} = kl (low-x reservoir) and th_n = thr,
 * kap_n = kr (high-x reservoir). The tridiagonal system is solved by Gaussian
 * elimination without pivoting (the Thomas algorithm; the matrix is strictly
 * diagonally dominant), then Er_p = delta rho_p th_p / 2.
 */
int ora_diffuse_be_line(int n, double delta, double dt, const double *rho, const double *kap,
                        double *Er, double thl, double kl, double thr, double kr)
{
    double *cp = (double *)malloc(sizeof(double) * n);
    double *rp = (double *)malloc(sizeof(double) * n);
    int p;
    if (!cp || !rp) {
        free(cp); free(rp);
        return 1;
    }
    for (p = 0; p < n; p++) {
        const double km = 0.5 * (kap[p] + (p > 0 ? kap[p - 1] : kl));
        const double kp = 0.5 * (kap[p] + (p < n - 1 ? kap[p + 1] : kr));
        const double a = p > 0 ? -dt * km : 0.0;
        const double c = p < n - 1 ? -dt * kp : 0.0;
        const double b = 0.5 * delta * rho[p] + dt * (km + kp);
        double r = Er[p];
        double m;
        if (p == 0) r += dt * km * thl;
        if (p == n - 1) r += dt * kp * thr;
        m = (p > 0) ? b - a * cp[p - 1] : b;
        cp[p] = c / m;
        rp[p] = (p > 0) ? (r - a * rp[p - 1]) / m : r / m;
    }
    for (p = n - 2; p >= 0; p--) rp[p] -= cp[p] * rp[p + 1]; /* rp now holds theta_R */
    for (p = 0; p < n; p++) Er[p] = 0.5 * delta * rho[p] * rp[p];
    free(cp); free(rp);
    return 0;
}

/*
 * nsteps time steps. Each step, in this order:
 *   1. collide every point (moments, recovery, targets, relaxation, and the
 *      rotational exchange), keeping rho, u and kappa_R of time t;
 *   2. pull-stream the populations;
 *   3. advect Er: MacCormack, forward differences in the predictor and
 *      backward differences in the corrector (Sec. 5, rotational step 2), in
 *      flux form F = Er v on each sublattice with axis neighbours at +-1. The
 *      advecting velocity is centred in time, v = (3 u(t) - u(t-1))/2, the
 *      second-order extrapolation to t + dt/2: in flux form the compression
 *      term -Er div v enters the linear acoustics, and v = u(t) would leave a
 *      first-order error there (a negative bulk viscosity of order dt);
 *      uprev (3 planes) holds u(t-1) on entry and u(t_end - 1) on return;
 * (rot_mode = 1 replaces 3 and 4 by the paper's four steps on theta_R, see
 * below.)
 *   4. diffuse: nsub FTCS sub-steps of dt/nsub of the flux-form equation
 *      dEr/dt = div(kappa_R grad theta_R), theta_R = 2 Er/(delta rho), face
 *      coefficients the mean of the two kappa_R values (Sec. 5, step 3, with
 *      eq. rotHeatFlux_simple; E_R = delta rho theta_R / 2, Sec. 3); with
 *      diff = 1 instead one backward-Euler step per sublattice line
 *      (ora_diffuse_be_line; quasi-1-D tubes only).
 * res (bcx = 1 only): 12 doubles, rho, ux, uy, uz, T, R of the low-x and then
 * the high-x reservoir.
 */
int ora_step(const ora_params *P, int nx, int ny, int nz, const double *res, double *g,
             double *Er, double *uprev, long nsteps)
{
    grid G = make_grid(nx, ny, nz);
    const long N = G.npts;
    double *gs = (double *)malloc(sizeof(double) * N * Q);
    double *rho = (double *)malloc(sizeof(double) * N);
    double *u = (double *)malloc(sizeof(double) * 3 * N);
    double *kap = (double *)malloc(sizeof(double) * N);
    double *Ep = (double *)malloc(sizeof(double) * N);
    double *Ec = (double *)malloc(sizeof(double) * N);
    double *th = (double *)malloc(sizeof(double) * N);
    double *v = (double *)malloc(sizeof(double) * 3 * N);
    double *Tt = (double *)malloc(sizeof(double) * N);
    double *rw = (double *)malloc(sizeof(double) * (2 * (long)nx * nz + 2 * (long)ny * nz));
    double gw[4][Q];
    ghost gh[6];
    long p, t;
    int i, a, k;
    if (!gs || !rho || !u || !kap || !Ep || !Ec || !th || !v || !Tt || !rw) {
        free(gs); free(rho); free(u); free(kap); free(Ep); free(Ec); free(th); free(v); free(Tt);
        free(rw);
        return 1;
    }
    need_lattice();
    if ((P->diff == 1 && (ny != 1 || nz != 1 || P->bcx != 1)) || (P->diff == 1 && P->rot_mode == 1) ||
        (P->bcy == 1 && (ny < 2 || P->bcx == 1 || P->diff == 1 ||
                         P->wall[1] != 0.0 || P->wall[5] != 0.0)) ||
        (P->bcx == 2 && (nx < 2 || P->diff == 1 || P->xwall[0] != 0.0 || P->xwall[4] != 0.0))) {
        free(gs); free(rho); free(u); free(kap); free(Ep); free(Ec); free(th); free(v); free(Tt);
        free(rw);
        return 2;
    }
    if (P->bcx == 1) {
        make_ghost(P, res, &gh[0]);
        make_ghost(P, res + 6, &gh[1]);
    }
    for (k = 0; k < 4; k++) {
        /* walls 0, 1: y (bcy = 1); walls 2, 3: x (bcx = 2) */
        const double *wl = (k < 2) ? P->wall + 4 * k : P->xwall + 4 * (k - 2);
        double Lam[9];
        if ((k < 2 && P->bcy != 1) || (k >= 2 && P->bcx != 2)) continue;
        for (a = 0; a < 9; a++) Lam[a] = (a % 4 == 0) ? wl[3] : 0.0;
        ora_target(1.0, wl, Lam, gw[k]);
        /* transport ghost: only u (the zero normal velocity) is read */
        gh[2 + k].rho = 1.0;
        gh[2 + k].Er = 0.5 * P->delta * wl[3];
        gh[2 + k].kap = 0.0;
        for (a = 0; a < 3; a++) gh[2 + k].u[a] = wl[a];
    }
    for (t = 0; t < nsteps; t++) {
        /* 1. collision and rotational exchange */
        for (p = 0; p < N; p++) {
            moments m;
            memcpy(gs + p * Q, g + p * Q, sizeof(double) * Q);
            collide(P, gs + p * Q, Er + p, &m);
            rho[p] = m.rho;
            for (a = 0; a < 3; a++) u[a * N + p] = m.u[a];
            kap[p] = kappa_R(P, m.rho, m.theta);
            Tt[p] = m.T;
        }
        /* 2. pull streaming; the walls emit rho_w f^eq(1, u_w, theta_w) */
        if ((P->bcy == 1 || P->bcx == 2) && wall_density(P, &G, gs, gw, rw)) {
            free(gs); free(rho); free(u); free(kap); free(Ep); free(Ec); free(th); free(v); free(Tt);
            free(rw);
            return 1;
        }
        for (p = 0; p < N; p++) {
            int x = (int)(p % nx), y = (int)((p / nx) % ny), z = (int)((p / ((long)nx * ny)) % nz);
            int s = (int)(p / G.n3);
            for (i = 0; i < Q; i++) {
                long q = pull_source(P, &G, s, x, y, z, i);
                if (q >= 0)
                    g[p * Q + i] = gs[q * Q + i];
                else if (q >= -2)
                    g[p * Q + i] = gh[-1 - q].g[i];
                else
                    g[p * Q + i] = rw[wall_slot(&G, (int)(-3 - q), x, y, z)] * gw[-3 - q][i];
            }
        }
        if (P->rot_mode == 1) {
            /* paper mode (Sec. 5, four steps on theta_R, held in Er[]), with
             * theta_T(f) of time t in both relaxation half steps */
            const double X = 3.0 * P->dt / (2.0 * P->tau1 * (3.0 + P->delta));
            /* 1. backward-Euler half step of the relaxation */
            for (p = 0; p < N; p++) Er[p] = (Er[p] + X * Tt[p]) / (1.0 + X);
            /* 2. MacCormack on u . grad theta_R: forward differences in the
             *    predictor, backward in the corrector, u of time t */
            for (p = 0; p < N; p++) {
                double adv = 0.0;
                for (a = 0; a < 3; a++) {
                    long qf = axis_nb(P, &G, p, a, +1);
                    double Rq = (qf >= 0) ? Er[qf]
                                : (qf >= -2) ? gh[-1 - qf].Er : wall_ghost(P, &G, p, qf, Er[p]);
                    adv += u[a * N + p] * (Rq - Er[p]);
                }
                Ep[p] = Er[p] - P->dt * adv;
            }
            for (p = 0; p < N; p++) {
                double adv = 0.0;
                for (a = 0; a < 3; a++) {
                    long qb = axis_nb(P, &G, p, a, -1);
                    double Rq = (qb >= 0) ? Ep[qb]
                                : (qb >= -2) ? gh[-1 - qb].Er : wall_ghost(P, &G, p, qb, Ep[p]);
                    adv += u[a * N + p] * (Ep[p] - Rq);
                }
                Ec[p] = 0.5 * (Er[p] + Ep[p] - P->dt * adv);
            }
            memcpy(Er, Ec, sizeof(double) * N);
            /* 3. FTCS of (2 / (rho delta)) kappa_R lap theta_R, nsub sub-steps */
            for (k = 0; k < P->nsub; k++) {
                const double h = P->dt / P->nsub;
                for (p = 0; p < N; p++) {
                    double lap = 0.0;
                    for (a = 0; a < 3; a++) {
                        long qp = axis_nb(P, &G, p, a, +1), qm = axis_nb(P, &G, p, a, -1);
                        double Rp = (qp >= 0) ? Er[qp]
                                    : (qp >= -2) ? gh[-1 - qp].Er : wall_ghost(P, &G, p, qp, Er[p]);
                        double Rm = (qm >= 0) ? Er[qm]
                                    : (qm >= -2) ? gh[-1 - qm].Er : wall_ghost(P, &G, p, qm, Er[p]);
                        lap += Rp - 2.0 * Er[p] + Rm;
                    }
                    Ec[p] = Er[p] + h * 2.0 * kap[p] / (rho[p] * P->delta) * lap;
                }
                memcpy(Er, Ec, sizeof(double) * N);
            }
            /* 4. second backward-Euler half step */
            for (p = 0; p < N; p++) Er[p] = (Er[p] + X * Tt[p]) / (1.0 + X);
            memcpy(uprev, u, sizeof(double) * 3 * N);
            continue;
        }
        /* 3. MacCormack advection of Er with v = (3 u(t) - u(t-1))/2 */
        for (p = 0; p < 3 * N; p++) v[p] = 1.5 * u[p] - 0.5 * uprev[p];
        memcpy(uprev, u, sizeof(double) * 3 * N);
        for (p = 0; p < N; p++) {
            double div = 0.0;
            for (a = 0; a < 3; a++) {
                long q = axis_nb(P, &G, p, a, +1);
                double Fq = (q >= 0) ? Er[q] * v[a * N + q] : gh[-1 - q].Er * gh[-1 - q].u[a];
                div += Fq - Er[p] * v[a * N + p];
            }
            Ep[p] = Er[p] - P->dt * div;
        }
        for (p = 0; p < N; p++) {
            double div = 0.0;
            for (a = 0; a < 3; a++) {
                long q = axis_nb(P, &G, p, a, -1);
                double Fq = (q >= 0) ? Ep[q] * v[a * N + q] : gh[-1 - q].Er * gh[-1 - q].u[a];
                div += Ep[p] * v[a * N + p] - Fq;
            }
            Ec[p] = 0.5 * (Er[p] + Ep[p] - P->dt * div);
        }
        memcpy(Er, Ec, sizeof(double) * N);
        /* 4. diffusion: backward Euler per sublattice line (variant) ... */
        if (P->diff == 1) {
            int sl;
            for (sl = 0; sl < 2; sl++) {
                const long o = (long)sl * nx;
                if (ora_diffuse_be_line(nx, P->delta, P->dt, rho + o, kap + o, Er + o,
                                        2.0 * gh[0].Er / (P->delta * gh[0].rho), gh[0].kap,
                                        2.0 * gh[1].Er / (P->delta * gh[1].rho), gh[1].kap)) {
                    free(gs); free(rho); free(u); free(kap); free(Ep); free(Ec); free(th); free(v);
                    free(Tt); free(rw);
                    return 1;
                }
            }
            continue;
        }
        /* ... or FTCS sub-steps */
        for (k = 0; k < P->nsub; k++) {
            const double h = P->dt / P->nsub;
            for (p = 0; p < N; p++) th[p] = 2.0 * Er[p] / (P->delta * rho[p]);
            for (p = 0; p < N; p++) {
                double acc = 0.0;
                for (a = 0; a < 3; a++) {
                    long qp = axis_nb(P, &G, p, a, +1), qm = axis_nb(P, &G, p, a, -1);
                    double thp = (qp >= 0) ? th[qp] : 2.0 * gh[-1 - qp].Er / (P->delta * gh[-1 - qp].rho);
                    double thm = (qm >= 0) ? th[qm] : 2.0 * gh[-1 - qm].Er / (P->delta * gh[-1 - qm].rho);
                    double kp = (qp >= 0) ? kap[qp] : gh[-1 - qp].kap;
                    double km = (qm >= 0) ? kap[qm] : gh[-1 - qm].kap;
                    if (qp <= -3 || qm <= -3) {
                        /* wall: face coefficient kappa_R(p), gradient over the
                         * distance d to the wall, as a ghost value on the axis
                         * neighbour (at distance 1 - d beyond the wall) */
                        const long qw = (qp <= -3) ? qp : qm;
                        const int w = (int)(-3 - qw), side = w & 1, s = (int)(p / G.n3);
                        const double *wl = (w < 2) ? P->wall : P->xwall;
                        const double d = wall_distance(s, side), thw = wl[4 * side + 3];
                        const double gv = thw + (thw - th[p]) * (1.0 - d) / d;
                        if (side == 1) { thp = gv; kp = kap[p]; } else { thm = gv; km = kap[p]; }
                    }
                    acc += 0.5 * (kap[p] + kp) * (thp - th[p]) - 0.5 * (kap[p] + km) * (th[p] - thm);
                }
                Ec[p] = Er[p] + h * acc;
            }
            memcpy(Er, Ec, sizeof(double) * N);
        }
    }
    free(gs); free(rho); free(u); free(kap); free(Ep); free(Ec); free(th); free(v); free(Tt);
    free(rw);
    return 0;
}

/* Hydrodynamic fields of the f-level state: rho, u (3 planes), theta_T(f),
 * theta_R and E_R = delta rho theta_R / 2. */
void ora_fields(const ora_params *P, int nx, int ny, int nz, const double *g, const double *Er,
                double *rho, double *u, double *T, double *R, double *ER)
{
    grid G = make_grid(nx, ny, nz);
    long p;
    int a;
    for (p = 0; p < G.npts; p++) {
        moments m;
        recover(P, g + p * Q, Er[p], &m);
        rho[p] = m.rho;
        for (a = 0; a < 3; a++) u[a * G.npts + p] = m.u[a];
        T[p] = m.T;
        R[p] = m.R;
        ER[p] = 0.5 * P->delta * m.rho * m.R;
    }
}

/*
 * Global diagnostics, summed in point order:
 *   out[0]   M  = sum rho
 *   out[1-3] J  = sum rho u
 *   out[4]   E  = sum (sum_i g_i c_i^2 / 2 + Er), equal to the f-level total
 *               E_T + E_R because the trapezoid shifts of the two cancel
 *   out[5]   H1 = sum [ sum_i (f_i ln(f_i/w_i) - f_i) - (delta/2) rho ln theta_R ]
 *               (Sec. 2 H function on the lattice, Sec. 4 H1 with k = -delta/2);
 *               NaN if some f_i <= 0
 *   out[6]   min_i,p g_i
 */
void ora_diag(const ora_params *P, int nx, int ny, int nz, const double *g, const double *Er,
              double *out)
{
    grid G = make_grid(nx, ny, nz);
    double M = 0.0, J[3] = {0.0, 0.0, 0.0}, E = 0.0, H = 0.0, gmin = INFINITY;
    long p;
    int i, a;
    need_lattice();
    for (p = 0; p < G.npts; p++) {
        double f[Q], c2, Hp = 0.0;
        moments m;
        const double *gp = g + p * Q;
        for (i = 0; i < Q; i++) {
            c2 = C[i][0] * C[i][0] + C[i][1] * C[i][1] + C[i][2] * C[i][2];
            M += gp[i];
            for (a = 0; a < 3; a++) J[a] += gp[i] * C[i][a];
            E += 0.5 * gp[i] * c2;
            if (gp[i] < gmin) gmin = gp[i];
        }
        f_from_g(P, gp, Er[p], f, &m);
        E += (P->rot_mode == 1) ? 0.5 * P->delta * m.rho * m.R : Er[p];
        for (i = 0; i < Q; i++) {
            if (f[i] <= 0.0) { Hp = NAN; break; }
            Hp += f[i] * log(f[i] / W[i]) - f[i];
        }
        H += Hp - 0.5 * P->delta * m.rho * log(m.R);
    }
    out[0] = M;
    for (a = 0; a < 3; a++) out[1 + a] = J[a];
    out[4] = E;
    out[5] = H;
    out[6] = gmin;
}
