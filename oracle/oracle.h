/*
 * FP64 CPU oracle for the 1D laser-foil PIC step with the leapfrog
 * Landau-Lifshitz radiation-reaction pusher of Tamburini et al.,
 * "Radiation Reaction Effects on Radiation Pressure Acceleration"
 * (arXiv 1008.1685).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library
 * against a plain, slow, obviously correct restatement of the method.  Only
 * the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  It shares no code, header, table or helper with the CUDA
 * library, and the CUDA library never calls it.
 *
 * Units (Sec. 2, after Eq. 3dLL): time in 1/omega, space in c/omega,
 * momenta in m_s c for species s, fields in m_e omega c/|e|, densities in
 * n_c.  Maxwell's equations read dE/dt = curl B - J, dB/dt = -curl E,
 * div E = rho.  One laser wavelength is 2*pi.
 *
 * Grid (1D Yee, x only): nodes i = 0..Nx carry Ey, Ez, Jy, Jz; half nodes
 * j = 0..Nx-1 at (j+1/2)dx carry Ex, By, Bz, Jx.  B is stored at integer
 * time (time-centred), E at integer time, momenta at half time.
 * Positions are stored as xi = x/dx (cell units).
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_sim or_sim;

typedef struct {
    double length_lambda;     /* box length in wavelengths */
    double cells_per_lambda;  /* dx = 2*pi / cells_per_lambda */
    double cfl;               /* dt/dx, 0 < cfl < 1 */
    double lambda_um;         /* laser wavelength in micrometres (sets eps) */
    int rr_on;                /* radiation reaction on electrons */
    int source_node;          /* node of the total-field/scattered-field plane */
} or_config;

/* ---- single particle (Sec. 3) ------------------------------------------ */

/* eps = (4/3) pi r_e / lambda (Eq. 3dLL), r_e in micrometres (CODATA). */
double or_eps_rr(double lambda_um);

/* One leapfrog step of the pusher of Sec. 3 for a particle of charge-to-mass
 * ratio qm (units e/m_e over m_s/m_e; -1 for electrons).  p (in m_s c) is
 * p^{n-1/2} on entry and p^{n+1/2} on return.  E, B are the fields at
 * (x^n, t^n).  rr != 0 adds the radiation-reaction kick of Eqs.
 * (f_r, pertfull, estim1, estimgamma); it is only meaningful for electrons.
 * Returns gamma(p_L) - gamma(p^{n+1/2}), the energy (in m_s c^2) removed by
 * the kick (0 without RR).  If pL is non-NULL it receives p_L^{n+1/2}. */
double or_push_boris_rr(double p[3], const double E[3], const double B[3],
                        double qm, double dt, double eps, int rr, double pL[3]);

/* Analytic plane waves travelling along +x with phase phi = t - x.
 *   kind 0: LP, Ey = a0 cos(phi)
 *   kind 1: CP, Ey = a0/sqrt2 cos(phi), Ez = a0/sqrt2 sin(phi)
 *   kind 2: LP, Ey = a0 sin^2(pi phi/tau) cos(phi) for 0<=phi<=tau, else 0
 * B = x_hat cross E, so By = -Ez, Bz = Ey. */
void or_planewave(int kind, double a0, double tau, double t, double x,
                  double E[3], double B[3], double dE[3]);

/* Electron (qm = -1) in a plane wave, Boris(+RR) leapfrog.  Initial data:
 * x^0 = x0 at t = 0, p^{-1/2} = p0.  Writes nout samples, one every `every`
 * steps starting after the first: out[k*5 + (0..4)] = t_n, x^n, then the
 * momentum p^{n-1/2} (3 values).  Returns 0 on success. */
int or_pw_leapfrog(int kind, double a0, double tau, double x0, const double p0[3],
                   double dt, int64_t nsteps, int every, double eps, int rr,
                   double* out, int64_t nout);

/* Electron in a plane wave, classical RK4 on Eq. (3dLL) in the lab frame.
 * deriv != 0 keeps the field-derivative term of Eq. (3dLL); rr == 0 drops
 * all radiation terms.  Initial data x(0) = x0, p(0) = p0; samples as
 * above but with t, x, p at the same time. */
int or_pw_rk4(int kind, double a0, double tau, double x0, const double p0[3],
              double dt, int64_t nsteps, int every, double eps, int rr, int deriv,
              double* out, int64_t nout);

/* ---- the 1D PIC (Sec. 3, Sec. 4) ----------------------------------------- */

or_sim* or_create(const or_config* cfg);
void or_destroy(or_sim* s);
int or_nx(const or_sim* s);
double or_dx(const or_sim* s);
double or_dt(const or_sim* s);

/* Uniform foil of both species, quiet start (electron k and ion k of a cell
 * share the in-cell offset), cold.  Offsets from SplitMix64 (see
 * pic_oracle.c).  ion_A is the mass number; Z = A = 1 means protons. */
int or_load_foil(or_sim* s, double x0_lambda, double thickness_lambda,
                 double ne_over_nc, int ion_Z, double ion_A, int ppc, uint64_t seed);

/* Explicit particles of one species (0 electrons, 1 ions).  weight is the
 * density each macro-particle carries (n_c), charge in e, mass in m_e. */
int or_load_particles(or_sim* s, int species, int64_t n, const int32_t* cell,
                      const double* off, const double* px, const double* py,
                      const double* pz, double weight, double charge, double mass);

/* Initial fields: Ey, Ez on Nx+1 nodes; Ex, By, Bz on Nx half nodes (B at
 * the same integer time as E). */
int or_set_fields(or_sim* s, const double* Ex, const double* Ey, const double* Ez,
                  const double* By, const double* Bz);

/* polarization 0 LP, 1 CP; envelope 0 sin^2 over duration, 1 trapezoid with
 * sin^2 rise and fall of rise_periods each. */
int or_inject_laser(or_sim* s, double a0, int polarization, int envelope,
                    double duration_periods, double rise_periods);

int or_step_n(or_sim* s, int64_t n);
int64_t or_steps_done(const or_sim* s);

/* out[6] = field energy of the accounting region, electron kinetic, ion
 * kinetic, radiated (cumulative), net Poynting flux in through the left
 * accounting plane (cumulative), Poynting flux out through the right plane
 * (cumulative).  Energies in m_e c^2 n_c (c/omega) per unit area. */
int or_energy(const or_sim* s, double out[6]);

/* Kinetic-energy spectrum in MeV, linear bins on [e_min, e_max):
 * counts[k] = sum of w*dx over particles in bin k divided by the bin width.
 * under_over (nullable) receives the same sums below e_min / at or above
 * e_max (not divided by a width). */
int or_spectra(const or_sim* s, int species, int nbins, double e_min, double e_max,
               double* counts, double* under_over);

/* Particle read-back in load order.  x in c/omega; flag 0 active, -1 left
 * the box through x=0, +1 through x=L.  Returns the count, or -1. */
int64_t or_read_particles(const or_sim* s, int species, int64_t cap, double* x,
                          double* px, double* py, double* pz, int32_t* flag);

/* Skin-layer observables of Sec. 4 (Figs. 2 and 4) per particle, in load
 * order, at the current step: the friction coefficient
 *   d = eps gamma^2 [E^2 - (v.E)^2 + v^2 B^2 - (v.B)^2 - 2 v.(E x B)]
 * of Eq. (damping), and the quantum parameter
 *   chi = gamma sqrt(E^2 - (v.E)^2 + v^2 B^2 - (v.B)^2 - 2 v.(E x B)) / E_cr,
 * E_cr = m c^2 / (hbar omega) in field units, whose plane-wave value for a
 * particle crossing the wave is the gamma sqrt(I/I_cr) of the classical
 * validity condition (Sec. 2).  Fields E^n, B^n gathered at x^n as the push
 * gathers them; v from the stored momentum p^{n-1/2}.  Frozen particles get
 * 0.  d, chi nullable.  Returns the count, or -1. */
int64_t or_snapshot(const or_sim* s, int species, int64_t cap, double* d, double* chi);

/* E_cr in field units m_e omega c/|e| for wavelength lambda_um. */
double or_ecr(double lambda_um);

/* comp: 0 Ex, 1 Ey, 2 Ez, 3 By, 4 Bz, 5 Jx, 6 Jy, 7 Jz (J of the last step).
 * Returns the number of values written, or -1. */
int64_t or_read_fields(const or_sim* s, int comp, int64_t cap, double* out);

#ifdef __cplusplus
}
#endif
#endif
