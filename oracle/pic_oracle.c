/*
 * FP64 CPU oracle: single-particle pushers and the 1D PIC of Tamburini et
 * al. (arXiv 1008.1685), written out step by step in the paper's order.
 *
 * TEST INFRASTRUCTURE ONLY: see oracle.h.  No blocking, fusion, sorting or
 * reordering beyond what the method states: particles are visited in load
 * order, the current is summed in that order, and the fields are advanced
 * node by node.  Every floating-point operation is IEEE double, round to
 * nearest (built with -ffp-contract=off so that no FMA changes a result).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846
#define OR_PAD 4 /* guard cells on each side of every grid array */

/* Classical electron radius in micrometres (CODATA 2018: 2.8179403262e-15 m).
 * The paper rounds it to 2.8e-9 um in Sec. 2 after Eq. (3dLL). */
#define OR_RE_UM 2.8179403262e-9
/* Electron rest energy in MeV (CODATA 2018). */
#define OR_MEC2_MEV 0.51099895000
/* Proton and atomic mass unit in electron masses (CODATA 2018). */
#define OR_MP_ME 1836.15267343
#define OR_MU_ME 1822.888486209

/* Reduced Compton wavelength hbar/(m_e c) in micrometres (CODATA 2018:
 * 3.8615926796e-13 m); the paper quotes 3.9e-7 um in Sec. 2. */
#define OR_LAMBDAC_UM 3.8615926796e-7

double or_eps_rr(double lambda_um) { return (4.0 / 3.0) * OR_PI * OR_RE_UM / lambda_um; }

/* E_cr = m^2 c^3/(hbar |e|) over the field unit m omega c/|e| is
 * m c^2/(hbar omega) = lambda / (2 pi hbar/(m c)). */
double or_ecr(double lambda_um) { return lambda_um / (2.0 * OR_PI * OR_LAMBDAC_UM); }

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* ------------------------------------------------------------------------ */
/* The pusher of Sec. 3.                                                     */
/* ------------------------------------------------------------------------ */

/* The radiation-reaction force of Eq. (f_r) for an electron with velocity v
 * in fields E, B:  f_R = -eps { f_L x B - (v.E) E + gamma^2 [f_L^2 - (v.E)^2] v },
 * f_L = -(E + v x B).  gamma is passed in (it is gamma^(n) of Eq. estimgamma). */
static void force_rr(const double v[3], double gamma, const double E[3], const double B[3],
                     double eps, double fR[3]) {
    double vxB[3], fL[3], fLxB[3];
    cross3(v, B, vxB);
    for (int k = 0; k < 3; k++) fL[k] = -(E[k] + vxB[k]);
    cross3(fL, B, fLxB);
    double vE = dot3(v, E);
    double bracket = gamma * gamma * (dot3(fL, fL) - vE * vE);
    for (int k = 0; k < 3; k++) fR[k] = -eps * (fLxB[k] - vE * E[k] + bracket * v[k]);
}

double or_push_boris_rr(double p[3], const double E[3], const double B[3], double qm, double dt,
                        double eps, int rr, double pL_out[3]) {
    /* Standard Boris step for the Lorentz force (Sec. 3, first paragraph):
     * half electric kick, magnetic rotation, half electric kick. */
    double h = 0.5 * qm * dt;
    double pm[3], t[3], s[3], pp[3], tmp[3], pL[3];
    for (int k = 0; k < 3; k++) pm[k] = p[k] + h * E[k];
    double gm = sqrt(1.0 + dot3(pm, pm));
    for (int k = 0; k < 3; k++) t[k] = h * B[k] / gm;
    double t2 = dot3(t, t);
    for (int k = 0; k < 3; k++) s[k] = 2.0 * t[k] / (1.0 + t2);
    cross3(pm, t, tmp);
    for (int k = 0; k < 3; k++) pp[k] = pm[k] + tmp[k];
    cross3(pp, s, tmp);
    for (int k = 0; k < 3; k++) pL[k] = pm[k] + tmp[k] + h * E[k];
    if (pL_out)
        for (int k = 0; k < 3; k++) pL_out[k] = pL[k];

    if (!rr) {
        for (int k = 0; k < 3; k++) p[k] = pL[k];
        return 0.0;
    }
    /* Eq. (estim1): p^(n) ~ (p_L^{n+1/2} + p^{n-1/2}) / 2, v^(n) = p^(n)/gamma^(n),
     * Eq. (estimgamma): gamma^(n) = sqrt(1 + p^(n)^2). */
    double pbar[3], v[3], fR[3];
    for (int k = 0; k < 3; k++) pbar[k] = 0.5 * (pL[k] + p[k]);
    double gbar = sqrt(1.0 + dot3(pbar, pbar));
    for (int k = 0; k < 3; k++) v[k] = pbar[k] / gbar;
    force_rr(v, gbar, E, B, eps, fR);
    /* Eq. (pertfull): p^{n+1/2} = p_L^{n+1/2} + f_R^(n) dt. */
    for (int k = 0; k < 3; k++) p[k] = pL[k] + dt * fR[k];
    return sqrt(1.0 + dot3(pL, pL)) - sqrt(1.0 + dot3(p, p));
}

/* ------------------------------------------------------------------------ */
/* Analytic plane waves for the single-particle checks of Sec. 3.            */
/* ------------------------------------------------------------------------ */

void or_planewave(int kind, double a0, double tau, double t, double x, double E[3], double B[3],
                  double dE[3]) {
    double phi = t - x;
    E[0] = E[1] = E[2] = 0.0;
    dE[0] = dE[1] = dE[2] = 0.0;
    if (kind == 0) {
        E[1] = a0 * cos(phi);
        dE[1] = -a0 * sin(phi);
    } else if (kind == 1) {
        double a = a0 / sqrt(2.0);
        E[1] = a * cos(phi);
        E[2] = a * sin(phi);
        dE[1] = -a * sin(phi);
        dE[2] = a * cos(phi);
    } else {
        if (phi >= 0.0 && phi <= tau) {
            double sn = sin(OR_PI * phi / tau), cs = cos(OR_PI * phi / tau);
            double g = sn * sn, dg = 2.0 * sn * cs * OR_PI / tau;
            E[1] = a0 * g * cos(phi);
            dE[1] = a0 * (dg * cos(phi) - g * sin(phi));
        }
    }
    /* B = x_hat x E */
    B[0] = 0.0;
    B[1] = -E[2];
    B[2] = E[1];
}

int or_pw_leapfrog(int kind, double a0, double tau, double x0, const double p0[3], double dt,
                   int64_t nsteps, int every, double eps, int rr, double* out, int64_t nout) {
    if (every <= 0 || dt <= 0.0 || nsteps < 0) return -1;
    double x = x0, p[3] = {p0[0], p0[1], p0[2]};
    double E[3], B[3], dE[3];
    int64_t k = 0;
    for (int64_t n = 0; n < nsteps; n++) {
        double t = (double)n * dt;
        or_planewave(kind, a0, tau, t, x, E, B, dE);
        or_push_boris_rr(p, E, B, -1.0, dt, eps, rr, NULL);
        double g = sqrt(1.0 + dot3(p, p));
        x += dt * p[0] / g;
        if ((n + 1) % every == 0 && k < nout) {
            double* o = out + 5 * k++;
            o[0] = (double)(n + 1) * dt;
            o[1] = x;
            o[2] = p[0];
            o[3] = p[1];
            o[4] = p[2];
        }
    }
    return 0;
}

/* Right-hand side of Eq. (3dLL) for an electron in a plane wave.
 * y = (x, px, py, pz).  The total derivative (d/dt + v.grad) of a field
 * that depends on t - x is (1 - v_x) d/dphi. */
static void ll_rhs(int kind, double a0, double tau, double t, const double y[4], double eps, int rr,
                   int deriv, double dy[4]) {
    double p[3] = {y[1], y[2], y[3]};
    double g = sqrt(1.0 + dot3(p, p));
    double v[3] = {p[0] / g, p[1] / g, p[2] / g};
    double E[3], B[3], dE[3], dB[3], vxB[3], F[3], FxB[3], vxdB[3];
    or_planewave(kind, a0, tau, t, y[0], E, B, dE);
    dB[0] = 0.0;
    dB[1] = -dE[2];
    dB[2] = dE[1];
    cross3(v, B, vxB);
    for (int k = 0; k < 3; k++) F[k] = E[k] + vxB[k]; /* E + v x B */
    double f[3];
    for (int k = 0; k < 3; k++) f[k] = -F[k];
    if (rr) {
        double vE = dot3(v, E);
        cross3(F, B, FxB);
        double bracket = g * g * (dot3(F, F) - vE * vE);
        for (int k = 0; k < 3; k++) f[k] += eps * (FxB[k] + vE * E[k]) - eps * bracket * v[k];
        if (deriv) {
            double s = 1.0 - v[0];
            cross3(v, dB, vxdB);
            for (int k = 0; k < 3; k++) f[k] -= eps * g * s * (dE[k] + vxdB[k]);
        }
    }
    dy[0] = v[0];
    dy[1] = f[0];
    dy[2] = f[1];
    dy[3] = f[2];
}

int or_pw_rk4(int kind, double a0, double tau, double x0, const double p0[3], double dt,
              int64_t nsteps, int every, double eps, int rr, int deriv, double* out, int64_t nout) {
    if (every <= 0 || dt <= 0.0 || nsteps < 0) return -1;
    double y[4] = {x0, p0[0], p0[1], p0[2]}, k1[4], k2[4], k3[4], k4[4], yt[4];
    int64_t k = 0;
    for (int64_t n = 0; n < nsteps; n++) {
        double t = (double)n * dt;
        ll_rhs(kind, a0, tau, t, y, eps, rr, deriv, k1);
        for (int i = 0; i < 4; i++) yt[i] = y[i] + 0.5 * dt * k1[i];
        ll_rhs(kind, a0, tau, t + 0.5 * dt, yt, eps, rr, deriv, k2);
        for (int i = 0; i < 4; i++) yt[i] = y[i] + 0.5 * dt * k2[i];
        ll_rhs(kind, a0, tau, t + 0.5 * dt, yt, eps, rr, deriv, k3);
        for (int i = 0; i < 4; i++) yt[i] = y[i] + dt * k3[i];
        ll_rhs(kind, a0, tau, t + dt, yt, eps, rr, deriv, k4);
        for (int i = 0; i < 4; i++) y[i] += dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
        if ((n + 1) % every == 0 && k < nout) {
            double* o = out + 5 * k++;
            o[0] = (double)(n + 1) * dt;
            for (int i = 0; i < 4; i++) o[1 + i] = y[i];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The 1D PIC.                                                               */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t n;
    double *xi, *px, *py, *pz; /* xi = x/dx; momenta in m_s c */
    int32_t* flag;             /* 0 active, -1 / +1 frozen at x = 0 / x = L */
    double w, q, m;            /* density per macro-particle (n_c), charge (e), mass (m_e) */
    int loaded;
} or_species;

struct or_sim {
    int Nx, is;
    double dx, dt, cfl, eps, lambda_um;
    int rr_on;
    double *mem, *Ex, *Ey, *Ez, *By, *Bz, *Jx, *Jy, *Jz;
    or_species sp[2];
    int laser, pol, env;
    double a0, tau, rise;
    int64_t step;
    double U_rad, U_in, U_out;
};

or_sim* or_create(const or_config* cfg) {
    if (!cfg) return NULL;
    if (!(cfg->cells_per_lambda > 0.0) || !(cfg->length_lambda > 0.0)) return NULL;
    if (!(cfg->cfl > 0.0 && cfg->cfl < 1.0) || !(cfg->lambda_um > 0.0)) return NULL;
    double ncell = cfg->length_lambda * cfg->cells_per_lambda;
    if (ncell < 8.0 || ncell > 1.0e9) return NULL;
    or_sim* s = (or_sim*)calloc(1, sizeof(or_sim));
    if (!s) return NULL;
    s->Nx = (int)llround(ncell);
    s->is = cfg->source_node;
    if (s->is < 2 || s->is > s->Nx - 4) {
        free(s);
        return NULL;
    }
    s->dx = 2.0 * OR_PI / cfg->cells_per_lambda;
    s->cfl = cfg->cfl;
    s->dt = cfg->cfl * s->dx;
    s->eps = or_eps_rr(cfg->lambda_um);
    s->lambda_um = cfg->lambda_um;
    s->rr_on = cfg->rr_on ? 1 : 0;
    size_t len = (size_t)s->Nx + 1 + 2 * OR_PAD;
    s->mem = (double*)calloc(8 * len, sizeof(double));
    if (!s->mem) {
        free(s);
        return NULL;
    }
    double** arr[8] = {&s->Ex, &s->Ey, &s->Ez, &s->By, &s->Bz, &s->Jx, &s->Jy, &s->Jz};
    for (int k = 0; k < 8; k++) *arr[k] = s->mem + k * len + OR_PAD;
    return s;
}

void or_destroy(or_sim* s) {
    if (!s) return;
    for (int k = 0; k < 2; k++) {
        free(s->sp[k].xi);
        free(s->sp[k].px);
        free(s->sp[k].py);
        free(s->sp[k].pz);
        free(s->sp[k].flag);
    }
    free(s->mem);
    free(s);
}

int or_nx(const or_sim* s) { return s->Nx; }
double or_dx(const or_sim* s) { return s->dx; }
double or_dt(const or_sim* s) { return s->dt; }
int64_t or_steps_done(const or_sim* s) { return s->step; }

static int species_alloc(or_species* sp, int64_t n) {
    size_t k = (size_t)(n > 0 ? n : 1);
    sp->xi = (double*)calloc(k, sizeof(double));
    sp->px = (double*)calloc(k, sizeof(double));
    sp->py = (double*)calloc(k, sizeof(double));
    sp->pz = (double*)calloc(k, sizeof(double));
    sp->flag = (int32_t*)calloc(k, sizeof(int32_t));
    if (!sp->xi || !sp->px || !sp->py || !sp->pz || !sp->flag) return -1;
    sp->n = n;
    sp->loaded = 1;
    return 0;
}

/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the n-th output of a
 * generator whose state starts at `seed` is mix(seed + n * golden_gamma). */
static uint64_t splitmix64_at(uint64_t seed, uint64_t n) {
    uint64_t z = seed + n * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

int or_load_foil(or_sim* s, double x0_lambda, double thickness_lambda, double ne_over_nc, int ion_Z,
                 double ion_A, int ppc, uint64_t seed) {
    if (!s || s->step > 0 || s->sp[0].loaded || s->sp[1].loaded) return -2;
    if (!(ne_over_nc > 0.0) || ion_Z < 1 || !(ion_A > 0.0) || ppc < 1) return -1;
    double cpl = 2.0 * OR_PI / s->dx;
    int64_t c0 = llround(x0_lambda * cpl);
    int64_t nc = llround(thickness_lambda * cpl);
    if (c0 < 0 || nc < 1 || c0 + nc > s->Nx) return -1;
    int64_t n = nc * (int64_t)ppc;
    if (n > 2147483647LL) return -1;
    for (int k = 0; k < 2; k++)
        if (species_alloc(&s->sp[k], n)) return -3;
    /* Electrons: q = -1, m = 1, weight ne/ppc.  Ions: charge Z, n_i = ne/Z. */
    s->sp[0].q = -1.0;
    s->sp[0].m = 1.0;
    s->sp[0].w = ne_over_nc / (double)ppc;
    s->sp[1].q = (double)ion_Z;
    s->sp[1].m = (ion_Z == 1 && ion_A == 1.0) ? OR_MP_ME : ion_A * OR_MU_ME;
    s->sp[1].w = ne_over_nc / ((double)ion_Z * (double)ppc);
    int64_t i = 0;
    for (int64_t c = c0; c < c0 + nc; c++) {
        for (int k = 0; k < ppc; k++, i++) {
            uint64_t r = splitmix64_at(seed, (uint64_t)c * (uint64_t)ppc + (uint64_t)k + 1ULL);
            double u = (double)(r >> 40) * (1.0 / 16777216.0); /* 24-bit dyadic offset */
            s->sp[0].xi[i] = (double)c + u;                       /* quiet start: same offset */
            s->sp[1].xi[i] = (double)c + u;
        }
    }
    return 0;
}

int or_load_particles(or_sim* s, int species, int64_t n, const int32_t* cell, const double* off,
                      const double* px, const double* py, const double* pz, double weight,
                      double charge, double mass) {
    if (!s || species < 0 || species > 1) return -1;
    if (s->step > 0 || s->sp[species].loaded) return -2;
    if (n < 0 || (n > 0 && (!cell || !off || !px || !py || !pz)) || !(mass > 0.0)) return -1;
    for (int64_t i = 0; i < n; i++)
        if (cell[i] < 0 || cell[i] >= s->Nx || !(off[i] >= 0.0 && off[i] < 1.0)) return -1;
    if (species_alloc(&s->sp[species], n)) return -3;
    or_species* sp = &s->sp[species];
    sp->w = weight;
    sp->q = charge;
    sp->m = mass;
    for (int64_t i = 0; i < n; i++) {
        sp->xi[i] = (double)cell[i] + off[i];
        sp->px[i] = px[i];
        sp->py[i] = py[i];
        sp->pz[i] = pz[i];
    }
    return 0;
}

int or_set_fields(or_sim* s, const double* Ex, const double* Ey, const double* Ez, const double* By,
                  const double* Bz) {
    if (!s) return -1;
    if (s->step > 0) return -2;
    for (int i = 0; i <= s->Nx; i++) {
        s->Ey[i] = Ey ? Ey[i] : 0.0;
        s->Ez[i] = Ez ? Ez[i] : 0.0;
    }
    for (int j = 0; j < s->Nx; j++) {
        s->Ex[j] = Ex ? Ex[j] : 0.0;
        s->By[j] = By ? By[j] : 0.0;
        s->Bz[j] = Bz ? Bz[j] : 0.0;
    }
    return 0;
}

int or_inject_laser(or_sim* s, double a0, int polarization, int envelope, double duration_periods,
                    double rise_periods) {
    if (!s) return -1;
    if (s->step > 0 || s->laser) return -2;
    if (!(a0 >= 0.0) || polarization < 0 || polarization > 1 || envelope < 0 || envelope > 1) return -1;
    if (!(duration_periods > 0.0)) return -1;
    if (envelope == 1 && !(rise_periods > 0.0 && 2.0 * rise_periods <= duration_periods)) return -1;
    s->laser = 1;
    s->a0 = a0;
    s->pol = polarization;
    s->env = envelope;
    s->tau = duration_periods * 2.0 * OR_PI;
    s->rise = rise_periods * 2.0 * OR_PI;
    return 0;
}

/* Field envelope g(s) of the incident pulse at retarded time s (Sec. 4:
 * sin^2 rise and fall; the sin^2-over-the-whole-pulse shape is the default). */
static double envelope(const or_sim* s, double t) {
    if (t < 0.0 || t > s->tau) return 0.0;
    if (s->env == 0) {
        double q = sin(OR_PI * t / s->tau);
        return q * q;
    }
    if (t < s->rise) {
        double q = sin(0.5 * OR_PI * t / s->rise);
        return q * q;
    }
    if (t > s->tau - s->rise) {
        double q = sin(0.5 * OR_PI * (s->tau - t) / s->rise);
        return q * q;
    }
    return 1.0;
}

/* Incident field components at retarded time t: Ey_inc = Bz_inc = ay,
 * Ez_inc = -By_inc = az.  a0 labels the intensity with the LP convention,
 * so each CP component carries a0/sqrt2. */
static void incident(const or_sim* s, double t, double* ay, double* az) {
    *ay = 0.0;
    *az = 0.0;
    if (!s->laser) return;
    double g = envelope(s, t);
    if (s->pol == 0) {
        *ay = s->a0 * g * sin(t);
    } else {
        double a = s->a0 / sqrt(2.0);
        *ay = a * g * sin(t);
        *az = -a * g * cos(t);
    }
}

static double half_val(const or_sim* s, const double* arr, int j) {
    return (j >= 0 && j < s->Nx) ? arr[j] : 0.0;
}

/* Linear-weight field gather at xi (Sec. 3: fields E^(n), B^(n) at the
 * particle; B here is the time-centred field). */
static void gather(const or_sim* s, double xi, double E[3], double B[3]) {
    double cf = floor(xi);
    int c = (int)cf;
    double f = xi - cf;
    E[1] = (1.0 - f) * s->Ey[c] + f * s->Ey[c + 1];
    E[2] = (1.0 - f) * s->Ez[c] + f * s->Ez[c + 1];
    double h = xi - 0.5;
    double jf = floor(h);
    int j = (int)jf;
    double g = h - jf;
    E[0] = (1.0 - g) * half_val(s, s->Ex, j) + g * half_val(s, s->Ex, j + 1);
    B[0] = 0.0;
    B[1] = (1.0 - g) * half_val(s, s->By, j) + g * half_val(s, s->By, j + 1);
    B[2] = (1.0 - g) * half_val(s, s->Bz, j) + g * half_val(s, s->Bz, j + 1);
}

static double shape(double xi, int i) {
    double d = fabs(xi - (double)i);
    return d < 1.0 ? 1.0 - d : 0.0;
}

/* Charge-conserving deposit of one particle moving from xi0 to xi1 (linear
 * shape): Jx_{k+1/2} = -(q w dx/dt) sum_{m<=k} [S_m(xi1) - S_m(xi0)], and
 * Jy,z on nodes with the time-averaged shape. */
static void deposit(or_sim* s, double a, double xi0, double xi1, double vy, double vz) {
    int c0 = (int)floor(xi0), c1 = (int)floor(xi1);
    int kmin = c0 < c1 ? c0 : c1;
    int kmax = (c0 > c1 ? c0 : c1) + 1;
    double jfac = -a * s->dx / s->dt, acc = 0.0;
    for (int k = kmin; k <= kmax; k++) {
        double s0 = shape(xi0, k), s1 = shape(xi1, k);
        s->Jy[k] += a * vy * 0.5 * (s0 + s1);
        s->Jz[k] += a * vz * 0.5 * (s0 + s1);
        acc += s1 - s0;
        if (k < kmax) s->Jx[k] += jfac * acc;
    }
}

/* Push and deposit particles i0 .. i1-1 of species k, in index order. */
static void push_range(or_sim* s, int k, int64_t i0, int64_t i1) {
    or_species* sp = &s->sp[k];
    double qm = sp->q / sp->m, a = sp->q * sp->w;
    int rr = (k == 0 && s->rr_on);
    for (int64_t i = i0; i < i1; i++) {
        if (sp->flag[i]) continue; /* frozen at a wall */
        double E[3], B[3], p[3] = {sp->px[i], sp->py[i], sp->pz[i]};
        double xi = sp->xi[i];
        gather(s, xi, E, B);
        double rad = or_push_boris_rr(p, E, B, qm, s->dt, s->eps, rr, NULL);
        s->U_rad += sp->w * s->dx * sp->m * rad;
        double g = sqrt(1.0 + dot3(p, p));
        double xn = xi + s->cfl * p[0] / g; /* x^{n+1} = x^n + dt v_x, in cell units */
        int fl = 0;
        if (xn < 0.0) {
            xn = 0.0;
            fl = -1;
        } else if (xn >= (double)s->Nx) {
            xn = (double)s->Nx;
            fl = 1;
        }
        deposit(s, a, xi, xn, p[1] / g, p[2] / g);
        sp->xi[i] = xn;
        sp->flag[i] = fl;
        sp->px[i] = p[0];
        sp->py[i] = p[1];
        sp->pz[i] = p[2];
    }
}

static void push_species(or_sim* s, int k) { push_range(s, k, 0, s->sp[k].n); }

#ifdef OR_PARALLEL_PUSH
static void push_species_parallel(or_sim* s, int k); /* pic_oracle_omp.c */
#endif

/* B half advance, B -= (dt/2) curl E, with the TF/SF correction at the last
 * scattered-field half node for the incident E at time t. */
static void b_half(or_sim* s, double t) {
    double hc = 0.5 * s->cfl;
    for (int j = 0; j < s->Nx; j++) {
        s->By[j] += hc * (s->Ez[j + 1] - s->Ez[j]);
        s->Bz[j] -= hc * (s->Ey[j + 1] - s->Ey[j]);
    }
    if (s->laser) {
        double ay, az;
        incident(s, t, &ay, &az); /* at node is: retarded time = t */
        int j = s->is - 1;
        s->Bz[j] += hc * ay;
        s->By[j] -= hc * az;
    }
}

static void field_step(or_sim* s) {
    int N = s->Nx, a = s->is + 1, b = N - 1;
    double c = s->cfl, dt = s->dt;
    double t0 = (double)s->step * dt;
    b_half(s, t0); /* B^n -> B^{n+1/2} */
    double ey0 = s->Ey[0], ey1 = s->Ey[1], eyn1 = s->Ey[N - 1], eyn = s->Ey[N];
    double ez0 = s->Ez[0], ez1 = s->Ez[1], ezn1 = s->Ez[N - 1], ezn = s->Ez[N];
    double eya = s->Ey[a], eza = s->Ez[a], eyb = s->Ey[b], ezb = s->Ez[b];
    for (int i = 1; i < N; i++) {
        s->Ey[i] += -c * (s->Bz[i] - s->Bz[i - 1]) - dt * s->Jy[i];
        s->Ez[i] += c * (s->By[i] - s->By[i - 1]) - dt * s->Jz[i];
    }
    if (s->laser) {
        double ay, az;
        /* incident B at half node is-1/2, time t0 + dt/2: retarded time t0 + dt/2 + dx/2 */
        incident(s, t0 + 0.5 * dt + 0.5 * s->dx, &ay, &az);
        s->Ey[s->is] += c * ay;
        s->Ez[s->is] += c * az;
    }
    /* First-order Mur absorbing ends. */
    double km = (c - 1.0) / (c + 1.0);
    s->Ey[0] = ey1 + km * (s->Ey[1] - ey0);
    s->Ez[0] = ez1 + km * (s->Ez[1] - ez0);
    s->Ey[N] = eyn1 + km * (s->Ey[N - 1] - eyn);
    s->Ez[N] = ezn1 + km * (s->Ez[N - 1] - ezn);
    for (int j = 0; j < N; j++) s->Ex[j] -= dt * s->Jx[j];
    /* Exact discrete Poynting flux through the accounting planes. */
    s->U_in += dt * (0.5 * (eya + s->Ey[a]) * s->Bz[a - 1] - 0.5 * (eza + s->Ez[a]) * s->By[a - 1]);
    s->U_out += dt * (0.5 * (eyb + s->Ey[b]) * s->Bz[b] - 0.5 * (ezb + s->Ez[b]) * s->By[b]);
    b_half(s, t0 + dt); /* B^{n+1/2} -> B^{n+1} */
}

int or_step_n(or_sim* s, int64_t n) {
    if (!s || n < 0) return -1;
    size_t len = (size_t)s->Nx + 1 + 2 * OR_PAD;
    for (int64_t it = 0; it < n; it++) {
        memset(s->Jx - OR_PAD, 0, len * sizeof(double));
        memset(s->Jy - OR_PAD, 0, len * sizeof(double));
        memset(s->Jz - OR_PAD, 0, len * sizeof(double));
        for (int k = 0; k < 2; k++) {
            if (!s->sp[k].loaded) continue;
#ifdef OR_PARALLEL_PUSH
            push_species_parallel(s, k);
#else
            push_species(s, k);
#endif
        }
        field_step(s);
        s->step++;
    }
    return 0;
}

static double kinetic(const or_species* sp, double dx) {
    double sum = 0.0;
    for (int64_t i = 0; i < sp->n; i++) {
        double p2 = sp->px[i] * sp->px[i] + sp->py[i] * sp->py[i] + sp->pz[i] * sp->pz[i];
        sum += p2 / (sqrt(1.0 + p2) + 1.0); /* gamma - 1 */
    }
    return sum * sp->w * dx * sp->m;
}

int or_energy(const or_sim* s, double out[6]) {
    if (!s || !out) return -1;
    int N = s->Nx, a = s->is + 1, b = N - 1;
    double hc = 0.5 * s->cfl, w = 0.0;
    for (int i = a; i <= b; i++) w += 0.5 * (s->Ey[i] * s->Ey[i] + s->Ez[i] * s->Ez[i]);
    for (int j = a; j <= b - 1; j++) {
        /* B^{n-1/2} . B^{n+1/2} = (B^n)^2 - ((dt/2) curl E^n)^2 */
        double dy = hc * (s->Ez[j + 1] - s->Ez[j]), dz = hc * (s->Ey[j + 1] - s->Ey[j]);
        w += 0.5 * (s->By[j] * s->By[j] - dy * dy + s->Bz[j] * s->Bz[j] - dz * dz);
    }
    for (int j = 0; j < N; j++) w += 0.5 * s->Ex[j] * s->Ex[j];
    out[0] = w * s->dx;
    out[1] = s->sp[0].loaded ? kinetic(&s->sp[0], s->dx) : 0.0;
    out[2] = s->sp[1].loaded ? kinetic(&s->sp[1], s->dx) : 0.0;
    out[3] = s->U_rad;
    out[4] = s->U_in;
    out[5] = s->U_out;
    return 0;
}

int or_spectra(const or_sim* s, int species, int nbins, double e_min, double e_max, double* counts,
               double* under_over) {
    if (!s || species < 0 || species > 1 || nbins < 1 || !(e_max > e_min) || !counts) return -1;
    const or_species* sp = &s->sp[species];
    double width = (e_max - e_min) / (double)nbins, uo[2] = {0.0, 0.0};
    for (int k = 0; k < nbins; k++) counts[k] = 0.0;
    for (int64_t i = 0; i < sp->n; i++) {
        double p2 = sp->px[i] * sp->px[i] + sp->py[i] * sp->py[i] + sp->pz[i] * sp->pz[i];
        double e = sp->m * OR_MEC2_MEV * p2 / (sqrt(1.0 + p2) + 1.0);
        double wt = sp->w * s->dx;
        if (e < e_min) {
            uo[0] += wt;
            continue;
        }
        double kf = floor((e - e_min) / (e_max - e_min) * (double)nbins);
        if (kf >= (double)nbins) {
            uo[1] += wt;
            continue;
        }
        counts[(int)kf] += wt;
    }
    for (int k = 0; k < nbins; k++) counts[k] /= width;
    if (under_over) {
        under_over[0] = uo[0];
        under_over[1] = uo[1];
    }
    return 0;
}

int64_t or_read_particles(const or_sim* s, int species, int64_t cap, double* x, double* px,
                          double* py, double* pz, int32_t* flag) {
    if (!s || species < 0 || species > 1) return -1;
    const or_species* sp = &s->sp[species];
    int64_t n = sp->n < cap ? sp->n : cap;
    for (int64_t i = 0; i < n; i++) {
        if (x) x[i] = sp->xi[i] * s->dx;
        if (px) px[i] = sp->px[i];
        if (py) py[i] = sp->py[i];
        if (pz) pz[i] = sp->pz[i];
        if (flag) flag[i] = sp->flag[i];
    }
    return sp->n;
}

int64_t or_snapshot(const or_sim* s, int species, int64_t cap, double* d, double* chi) {
    if (!s || species < 0 || species > 1) return -1;
    const or_species* sp = &s->sp[species];
    const double ecr = or_ecr(s->lambda_um);
    int64_t n = sp->n < cap ? sp->n : cap;
    for (int64_t i = 0; i < n; i++) {
        double dv = 0.0, cv = 0.0;
        if (!sp->flag[i]) {
            double E[3], B[3], p[3] = {sp->px[i], sp->py[i], sp->pz[i]};
            gather(s, sp->xi[i], E, B);
            double g = sqrt(1.0 + dot3(p, p));
            double v[3] = {p[0] / g, p[1] / g, p[2] / g};
            double ExB[3];
            cross3(E, B, ExB);
            double vE = dot3(v, E), vB = dot3(v, B);
            /* the bracket of Eq. (damping), first form */
            double br = dot3(E, E) - vE * vE + dot3(v, v) * dot3(B, B) - vB * vB - 2.0 * dot3(v, ExB);
            if (br < 0.0) br = 0.0; /* >= 0 exactly; rounding only */
            dv = s->eps * g * g * br;
            cv = g * sqrt(br) / ecr;
        }
        if (d) d[i] = dv;
        if (chi) chi[i] = cv;
    }
    return sp->n;
}

int64_t or_read_fields(const or_sim* s, int comp, int64_t cap, double* out) {
    if (!s || comp < 0 || comp > 7 || !out) return -1;
    const double* src[8] = {s->Ex, s->Ey, s->Ez, s->By, s->Bz, s->Jx, s->Jy, s->Jz};
    int node = (comp == 1 || comp == 2 || comp == 6 || comp == 7);
    int64_t n = node ? s->Nx + 1 : s->Nx;
    if (cap < n) return -1;
    for (int64_t i = 0; i < n; i++) out[i] = src[comp][i];
    return n;
}
