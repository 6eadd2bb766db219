/*
 * picrr — GB300-native (sm_103a) 1D laser-foil particle-in-cell step with
 * the leapfrog Landau-Lifshitz radiation-reaction pusher of Tamburini et
 * al., "Radiation Reaction Effects on Radiation Pressure Acceleration"
 * (arXiv 1008.1685).
 *
 * One time step is: linear field gather, Boris push plus the LL
 * radiation-reaction kick of Sec. 3 (Eqs. f_r, pertfull, estim1,
 * estimgamma), charge-conserving current deposit, 1D Yee update of Ex, Ey,
 * Ez, By, Bz with total-field/scattered-field laser injection and Mur
 * absorbing ends, and a periodic cell sort of the particles.
 *
 * Units (Sec. 2, after Eq. 3dLL): time 1/omega, length c/omega, momentum
 * m_s c of species s, fields m_e omega c/|e|, densities n_c.  One laser
 * wavelength is 2*pi; dx = 2*pi / cells_per_lambda, dt = cfl * dx.
 *
 * Grid: nodes i = 0..Nx at x = i*dx carry Ey, Ez, Jy, Jz; half nodes
 * j = 0..Nx-1 at (j+1/2)*dx carry Ex, By, Bz, Jx.  E and B are reported at
 * integer time (B is the time-centred field the particles see); momenta
 * at half time.
 *
 * Conventions for every entry point:
 *  - Return PIC_OK (0) or a negative pic_status.  A call that fails leaves
 *    the simulation unchanged, except pic_step_n, which may stop early and
 *    then reports the steps completed in *steps_done; the state is then
 *    consistent at that step.  pic_last_error() describes the last failure.
 *  - All array arguments are HOST pointers owned by the caller; the library
 *    copies what it needs before returning.  The library owns all device
 *    memory it allocates and frees it in pic_destroy.
 *  - A handle may be used by one thread at a time.  The library keeps no
 *    global mutable state; handles are independent.
 *  - Call order: pic_create, then any of pic_load_foil / pic_load_particles
 *    / pic_set_fields / pic_inject_laser (each at most once, and only before
 *    the first step), then pic_step_n any number of times.  Read-outs are
 *    allowed at any time.  Other orders return PIC_ERR_STATE.
 */
#ifndef PICRR_H
#define PICRR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic_sim pic_sim;

typedef enum {
    PIC_OK = 0,
    PIC_ERR_INVALID_ARG = -1,
    PIC_ERR_STATE = -2,
    PIC_ERR_OOM = -3,
    PIC_ERR_CUDA = -4,
    PIC_ERR_TIMEOUT = -5,
    PIC_ERR_UNSUPPORTED = -6
} pic_status;

enum { PIC_LP = 0, PIC_CP = 1 };
enum { PIC_ENV_SIN2 = 0, PIC_ENV_TRAPEZOID = 1 };
enum { PIC_ELECTRON = 0, PIC_ION = 1 };
enum { PIC_EX = 0, PIC_EY = 1, PIC_EZ = 2, PIC_BY = 3, PIC_BZ = 4, PIC_JX = 5, PIC_JY = 6, PIC_JZ = 7 };

/* Run configuration (Sec. 4: 1D box, laser wavelength lambda = 0.8 um). */
typedef struct {
    double length_lambda;    /* box length L in wavelengths, > 0 */
    double cells_per_lambda; /* grid resolution; Nx = round(L * cells_per_lambda) >= 16 */
    double cfl;              /* dt/dx, 0 < cfl < 1 (a particle moves < 1 cell per step) */
    double lambda_um;        /* wavelength in micrometres; sets eps = (4/3) pi r_e / lambda */
    int rr_on;               /* 1: radiation-reaction kick on electrons (Sec. 3); 0: Boris only */
    int sort_interval;       /* steps between cell sorts, 1..96 (0 selects 8) */
    uint64_t seed;           /* seed of the foil loader's counter-based generator */
    int device;              /* CUDA device ordinal */
    int source_node;         /* node of the laser injection plane, 2..Nx-4 (0 selects 8) */
    size_t hbm_budget_bytes; /* device memory limit for this handle, 0 = no limit */
} pic_config;

/* Create a run: allocates the grid (fields, currents) on cfg->device.
 * *out is set to NULL on error.  PIC_ERR_OOM if the grid exceeds the budget. */
pic_status pic_create(const pic_config* cfg, pic_sim** out);

/* Launch all work of this handle on the given cudaStream_t (NULL restores
 * the handle's own stream).  The stream must belong to the handle's device
 * and outlive its use.  Host calls still synchronise before returning. */
pic_status pic_set_stream(pic_sim* sim, void* cuda_stream);

/* Uniform foil of both species (Sec. 4): electrons (charge -1, mass m_e)
 * and ions of charge ion_Z and mass number ion_A (Z = A = 1: protons,
 * m_p = 1836.15267343 m_e; otherwise A * 1822.888486209 m_e), density
 * ne_over_nc electrons per n_c, occupying [x0, x0 + thickness] (in
 * wavelengths, rounded to whole cells), ppc macro-particles per cell per
 * species, cold.  Quiet start: electron k and ion k of a cell share the
 * in-cell offset u = (SplitMix64(seed, cell*ppc + k + 1) >> 40) * 2^-24.
 * Weights: ne/ppc (electrons), ne/(Z*ppc) (ions). */
pic_status pic_load_foil(pic_sim* sim, double x0_lambda, double thickness_lambda, double ne_over_nc,
                         int ion_Z, double ion_A, int ppc);

/* Explicit particles of one species (test and restart path).  cell[n] in
 * [0, Nx), off[n] in [0,1) is the in-cell offset, px/py/pz in m_s c; all
 * are rounded to float.  weight: density per macro-particle (n_c); charge
 * in e; mass in m_e.  Species PIC_ELECTRON gets the radiation-reaction
 * kick when rr_on is set.  n <= 2^31 - 1. */
pic_status pic_load_particles(pic_sim* sim, int species, int64_t n, const int32_t* cell,
                              const double* off, const double* px, const double* py,
                              const double* pz, double weight, double charge, double mass);

/* Same as pic_load_particles with single-precision host arrays, copied as
 * they are (no conversion).  When cell[] is already non-decreasing the five
 * arrays go straight to the device with asynchronous copies (pin them for
 * full bandwidth) and ids are generated on the device; otherwise the library
 * first makes a cell-ordered host copy. */
pic_status pic_load_particles_f32(pic_sim* sim, int species, int64_t n, const int32_t* cell,
                                  const float* off, const float* px, const float* py, const float* pz,
                                  double weight, double charge, double mass);

/* Initial fields (default all zero): Ey, Ez on Nx+1 nodes; Ex, By, Bz on Nx
 * half nodes; B at the same integer time as E.  Any pointer may be NULL
 * (that component stays zero). */
pic_status pic_set_fields(pic_sim* sim, const double* Ex, const double* Ey, const double* Ez,
                          const double* By, const double* Bz);

/* Laser entering at the source node, travelling towards +x (Sec. 4).
 * a0 labels the intensity with the LP convention (I lambda^2 =
 * 1.37e18 a0^2 W cm^-2 um^2), so CP has a0/sqrt2 per component.
 * LP: Ey = Bz = a0 g(s) sin(s); CP: Ey = Bz = a0/sqrt2 g sin(s),
 * Ez = -By = -a0/sqrt2 g cos(s); s = t - (x - x_source).
 * PIC_ENV_SIN2: g = sin^2(pi s / tau), tau = duration_periods * 2 pi.
 * PIC_ENV_TRAPEZOID: sin^2 rise and fall of rise_periods each, flat
 * between, total duration_periods (the shape of Sec. 4). */
pic_status pic_inject_laser(pic_sim* sim, double a0, int polarization, int envelope,
                            double duration_periods, double rise_periods);

/* Advance n >= 0 steps.  Synchronous: returns after the device has
 * finished; *steps_done (nullable) receives the steps completed in this
 * call.  PIC_ERR_TIMEOUT if a bounded device wait gave up (the state is
 * then that of the last completed step). */
pic_status pic_step_n(pic_sim* sim, int64_t n, int64_t* steps_done);

/* Kinetic-energy spectrum of one species, E = m_s c^2 (gamma - 1) in MeV,
 * nbins linear bins over [e_min, e_max): counts[k] = sum of w*dx over
 * particles in bin k divided by the bin width (dN/dE per unit area, in
 * n_c c/omega per MeV).  Particles that left the box are included.
 * radiated_J_per_m2 (nullable) receives the energy removed by radiation
 * reaction so far, in J per m^2 of transverse area. */
pic_status pic_spectra(pic_sim* sim, int species, int nbins, double e_min_MeV, double e_max_MeV,
                       double* counts, double* radiated_J_per_m2);

/* out[6], energies per unit area in m_e c^2 n_c c/omega (FP64):
 *  [0] field energy of the accounting region (nodes source+1..Nx-1; B
 *      enters as B^{n-1/2}.B^{n+1/2}, the quantity the Yee scheme conserves),
 *  [1] electron kinetic energy, [2] ion kinetic energy (momenta at n-1/2),
 *  [3] energy radiated by the kick so far, w*dx*(gamma(p_L) - gamma(p)),
 *  [4] net Poynting flux in through the left accounting plane so far,
 *  [5] Poynting flux out through the right accounting plane so far. */
pic_status pic_energy(pic_sim* sim, double out[6]);

/* Particle read-back in load order.  x in c/omega, momenta in m_s c,
 * flag 0 active, -1 / +1 frozen at x = 0 / x = L.  Arrays (each nullable)
 * hold at least cap entries; *n (nullable) receives the species count. */
pic_status pic_read_particles(pic_sim* sim, int species, int64_t cap, double* x, double* px,
                              double* py, double* pz, int32_t* flag, int64_t* n);

/* One grid component (PIC_EX..PIC_JZ; J of the last step): Nx+1 node values
 * or Nx half-node values; *n (nullable) receives the count. */
pic_status pic_read_fields(pic_sim* sim, int comp, int64_t cap, double* out, int64_t* n);

/* Skin-layer snapshot of Sec. 4 (Figs. 2 and 4) for one species at the
 * current step, computed on the device: per particle the friction
 * coefficient d = eps gamma^2 [f_L^2 - (v.f_L)^2] of Eq. (damping) (the
 * strength of the RR force in units of m omega c) and the quantum parameter
 * chi = gamma sqrt(f_L^2 - (v.f_L)^2) / E_cr, E_cr = m c^2/(hbar omega) in
 * field units (for a particle crossing a plane wave this is the
 * gamma sqrt(I/I_cr) of the classical validity condition of Sec. 2; the
 * classical treatment needs chi << 1).  Both are evaluated from the stored
 * momentum p^{n-1/2} and the fields E^n, B^n interpolated at x^n as the push
 * interpolates them; frozen particles give 0.  summary (nullable, [3]):
 * max d, max chi, number of particles with chi >= chi_flag (chi_flag >= 0).
 * With cap > 0, x (c/omega), p_x, p_perp = sqrt(p_y^2 + p_z^2), d and chi
 * (each nullable) receive the values of the first cap particles in load
 * order, as pic_read_particles.  *n (nullable) receives the species count. */
pic_status pic_snapshot(pic_sim* sim, int species, double chi_flag, int64_t cap, double* x, double* px,
                        double* pperp, double* d, double* chi, double* summary, int64_t* n);

typedef struct {
    int64_t steps;            /* steps completed since creation */
    int64_t kernel_launches;  /* device kernels launched by this handle */
    int64_t push_launches;    /* launches of the fused gather/push/deposit kernel */
    int64_t sort_count;       /* cell sorts performed */
    int64_t active_particles; /* particles of the runs still stepping, both species (frozen ones included) */
    double push_ms;           /* summed device time of the push kernel (timing on) */
    double field_ms;          /* summed device time of the Yee kernel (timing on) */
    double sort_ms;           /* summed device time of the sort kernels (timing on) */
    int64_t timed_push_launches; /* push launches covered by push_ms */
    int64_t device_bytes;     /* device memory held by the handle */
    int32_t n_units;          /* current work units (sorted particle chunks) */
    int32_t fp_bits;          /* fixed-point fraction bits of the current accumulators */
    int64_t graph_launches;   /* CUDA-graph launches, each one sort interval of steps */
    int32_t steps_since_sort; /* steps since the last cell sort (the next sort comes after
                                 sort_interval - steps_since_sort more steps) */
    int32_t reserved;
} pic_stats_t;

/* Launch shapes.  unit_particles: the most particles one CTA of the fused
 * push kernel takes (its work unit), a power of two in [1024, 16384]
 * (default 4096); sort_interval in [1, 96]; particles_per_thread: 4 or 2,
 * the particles each thread of the push kernel takes per round (4: 128-bit
 * loads and stores and the fewest instructions per particle, for dense foils;
 * 2: fewer registers and more warps per SM, which hides the latency of
 * deposits that scatter over many cells; default 2, so that a run gives the
 * same bits alone and in a batch; the tuner picks 4 for dense foils).  Larger units amortise each CTA's fixed costs on dense foils;
 * smaller ones keep the GPU busy when few particles are spread thinly.  A new
 * unit size takes effect at once (the run is sorted if needed and its unit
 * table rebuilt).  None of them changes more than the order of
 * single-precision sums. */
pic_status pic_set_shapes(pic_sim* sim, int unit_particles, int sort_interval, int particles_per_thread);

/* Shape tuner.  Steps the run for a trial of about steps_per_candidate steps
 * (rounded to whole sort intervals, after one warm-up interval) with 4 and 2
 * particles per thread, keeps the faster, then at each unit size of {2048,
 * 4096, 8192, 16384}, keeps the fastest, then at each sort interval of {8, 16,
 * 32, 64, 96}; measures the wall time per step (CUDA graphs, as pic_step_n
 * runs them) and keeps the fastest shapes.  *unit_particles, *sort_interval and
 * *particles_per_thread (nullable) receive them; ms_per_step[11] (nullable)
 * the measured times per step (particles per thread 4, 2; unit sizes;
 * intervals; -1 where not measured).  The trial steps are real steps of the
 * run.  Timing must be off. */
pic_status pic_tune_shapes(pic_sim* sim, int64_t steps_per_candidate, int* unit_particles, int* sort_interval,
                           int* particles_per_thread, double* ms_per_step);

/* Counters and, when timing is on, CUDA-event times of each kernel class,
 * recorded on the launching stream.  Every whole sort interval of steps that
 * no run ends inside is launched as one captured CUDA graph (its pushes, Yee
 * updates and the sort); with timing on, that graph also holds an event-record
 * node before and after each push, Yee update and sort, and the other steps
 * record their events around each launch.  The times are read when a step
 * call returns (and before a graph is launched again). */
pic_status pic_stats(pic_sim* sim, pic_stats_t* out);
pic_status pic_set_timing(pic_sim* sim, int on);

/* Switch the radiation-reaction kick of the electrons (Sec. 3, Eqs. f_r and
 * pertfull) on (1) or off (0) from the next step on; the rest of the state is
 * kept.  With it off the push is the Boris pusher alone.  It exists to
 * measure what the kick costs on one and the same state (the paper puts the
 * extra computing time at about 10 %, Sec. 3 last paragraph); the kick is
 * evaluated for every electron whenever it is on, whatever the field.
 * PIC_ERR_INVALID_ARG unless rr_on is 0 or 1. */
pic_status pic_set_rr(pic_sim* sim, int rr_on);

/* Message for the last failed call on sim (or on creation when sim is NULL,
 * for the calling thread).  Valid until the next call on the handle. */
const char* pic_last_error(const pic_sim* sim);

/* Free everything; NULL is accepted. */
pic_status pic_destroy(pic_sim* sim);

/* Checkpoint: write the run's complete state (fields of the current step,
 * the last step's current, particles in cell order with their ids, species
 * constants, laser, energy tallies, step count) to a binary file at path.  If
 * particles moved since the last sort, the run is sorted first (that changes
 * only the order of single-precision sums of later steps).  pic_restore
 * creates a new handle on `device` in that state (sort_interval as in
 * pic_config, 0 selects 8); stepping it continues the run: saved on a sort
 * step, the continuation is bit-identical to the uninterrupted run. */
pic_status pic_save(pic_sim* sim, const char* path);
/* The configuration of a handle (as created or restored; sort_interval current). */
pic_status pic_get_config(const pic_sim* sim, pic_config* out);
pic_status pic_restore(const char* path, int device, int sort_interval, pic_sim** out);

/* Self-test of failure detection on the device: launches one small kernel
 * whose mbarrier wait can never complete (it expects two arrivals and gets
 * one).  The wait is the bounded one every kernel of this library uses; it
 * gives up after its fixed number of polls, the kernel records the timeout in
 * a status word and the call returns PIC_ERR_TIMEOUT, with the CUDA context
 * still usable.  *seconds (nullable) receives the wall time it took.  No
 * trap, fault or unbounded wait is involved. */
pic_status pic_selftest_wait_timeout(int device, double* seconds);

/* ---- Batches of independent runs ---------------------------------------------
 * A batch steps many independent runs together: every kernel of a step is
 * one launch for all active runs of the batch, so small runs share the GPU
 * instead of each leaving most of it idle.  All runs of a batch share the
 * grid resolution, cfl, wavelength and sort interval of the batch's
 * pic_config (its length_lambda, rr_on, seed and source_node are unused);
 * everything else is per run.  Each run gives the same results alone and in
 * a batch (up to single-precision rounding: the batch changes no arithmetic
 * of a run, only how its work is packed into launches).  A pic_sim handle is
 * a batch of one run. */
typedef struct pic_batch pic_batch;

/* One run: box, foil (as pic_load_foil), laser (as pic_inject_laser), length. */
typedef struct {
    double length_lambda;  /* box length in wavelengths */
    int source_node;       /* laser injection node, 0 selects 8 */
    int rr_on;             /* radiation reaction on electrons */
    uint64_t seed;         /* foil loader seed */
    double foil_x0_lambda, foil_thickness_lambda, ne_over_nc;
    int ion_Z;
    double ion_A;
    int ppc;
    double a0;
    int polarization, envelope;
    double duration_periods, rise_periods;
    int64_t steps;         /* the run stops after this many steps (>= 1) */
} pic_run_desc;

/* Batch with room for max_runs runs (1..8192) on common->device. */
pic_status pic_batch_create(const pic_config* common, int max_runs, pic_batch** out);
/* As pic_set_stream. */
pic_status pic_batch_set_stream(pic_batch* batch, void* cuda_stream);
/* Add a run (allocates its grid and particles, generates its foil).  It joins
 * the batch at the next pic_batch_step, at a sort boundary (the batch sorts
 * early if needed).  *run_id receives its slot.  PIC_ERR_OOM if the budget is
 * exceeded (the batch is unchanged); PIC_ERR_STATE if all slots are used. */
pic_status pic_batch_add_run(pic_batch* batch, const pic_run_desc* desc, int* run_id);
/* Advance every active run by up to n steps; a run stops when it reaches its
 * own step count.  *steps_done (nullable) receives the batch steps taken (0
 * when no run is active).  Synchronous. */
pic_status pic_batch_step(pic_batch* batch, int64_t n, int64_t* steps_done);
/* Steps completed by a run and whether it has finished. */
pic_status pic_batch_run_status(pic_batch* batch, int run, int64_t* steps_done, int* finished);
/* Per-run read-outs, as pic_energy / pic_spectra / pic_read_particles / pic_read_fields. */
pic_status pic_batch_energy(pic_batch* batch, int run, double out[6]);
pic_status pic_batch_spectra(pic_batch* batch, int run, int species, int nbins, double e_min_MeV,
                             double e_max_MeV, double* counts, double* radiated_J_per_m2);
pic_status pic_batch_read_particles(pic_batch* batch, int run, int species, int64_t cap, double* x,
                                    double* px, double* py, double* pz, int32_t* flag, int64_t* n);
pic_status pic_batch_read_fields(pic_batch* batch, int run, int comp, int64_t cap, double* out, int64_t* n);
/* As pic_snapshot, for one run of the batch. */
pic_status pic_batch_snapshot(pic_batch* batch, int run, int species, double chi_flag, int64_t cap, double* x,
                              double* px, double* pperp, double* d, double* chi, double* summary, int64_t* n);
/* Stop a run before its step count (between steps): it leaves the batch at
 * its current step, and its state stays readable until released. */
pic_status pic_batch_stop_run(pic_batch* batch, int run);
/* Free a finished, stopped or not yet started run's device memory; its slot can take a new run. */
pic_status pic_batch_release_run(pic_batch* batch, int run);
/* Device bytes the run described by desc would take in this batch: its grid,
 * sort scratch and both particle buffers, plus its share of the batch's work
 * unit table with that table's growth headroom.  No allocation; used for
 * admission by memory.  Reads only the batch's configuration, so it may be
 * called from any thread; its error message is pic_batch_last_error(NULL). */
pic_status pic_batch_run_footprint(const pic_batch* batch, const pic_run_desc* desc, size_t* bytes);

/* Split independent runs over n_ranks GPUs, one process (rank) per GPU.  The
 * paper has no counterpart: it is the scheduling of a scan or a request stream
 * of independent runs.  Host only (no device call).  The work of a run is its
 * particle-steps (both species: 2 * ppc * cells of the foil * steps); each run
 * goes to the rank with the least work assigned so far among those whose
 * assigned footprints (pic_batch_run_footprint for common->cells_per_lambda,
 * summed, as if all runs of a rank were resident at once) stay within
 * budget_per_rank bytes (0: no limit); ties go to the lowest rank.
 * in_order = 0: runs taken in decreasing order of work (a scan known in
 * advance); in_order = 1: in the given order (a request stream, assigned as
 * the requests arrive).  The result depends only on the arguments, so every
 * rank computes the same assignment without exchanging anything.
 * rank_of_run[n_runs] receives the rank of each run; work_per_rank[n_ranks]
 * (nullable) the particle-steps assigned to each rank.  PIC_ERR_OOM (nothing
 * written) if a run fits no rank; errors are reported by pic_last_error(NULL). */
pic_status pic_shard_runs(const pic_config* common, const pic_run_desc* runs, int n_runs, int n_ranks,
                          int in_order, size_t budget_per_rank, int* rank_of_run, double* work_per_rank);
/* As pic_set_shapes / pic_tune_shapes, for all active runs of the batch together. */
pic_status pic_batch_set_shapes(pic_batch* batch, int unit_particles, int sort_interval, int particles_per_thread);
pic_status pic_batch_tune_shapes(pic_batch* batch, int64_t steps_per_candidate, int* unit_particles,
                                 int* sort_interval, int* particles_per_thread, double* ms_per_step);
pic_status pic_batch_stats(pic_batch* batch, pic_stats_t* out);
pic_status pic_batch_set_timing(pic_batch* batch, int on);
const char* pic_batch_last_error(const pic_batch* batch);
pic_status pic_batch_destroy(pic_batch* batch);

/* ---- Serving: a request loop over a batch --------------------------------
 * A server owns one batch and one worker thread.  Run requests are queued
 * when submitted and admitted (in arrival order by default, see
 * pic_server_set_policy) while a batch slot is free and
 * the run's footprint (pic_batch_run_footprint) fits the device-memory
 * budget (hbm_budget_bytes of the pic_config; 0: no budget).  Admitted runs
 * join the running batch between step chunks (continuous batching: a request
 * that arrives while others are stepping starts without waiting for them),
 * stay resident on the device until their last step, and the worker then
 * computes their ion and electron spectra and energy read-outs, frees their
 * memory and admits more.  Results stay in the server until fetched.
 * Each result is the same as that of the run stepped alone (see the batch
 * above).  All calls are thread-safe. */
typedef struct pic_server pic_server;

typedef struct {
    int64_t submitted, admitted, completed, failed;
    int64_t queued, running;      /* now */
    int64_t batch_steps;          /* steps taken by the batch */
    int64_t particle_steps;       /* particles pushed, summed over steps and runs */
    double busy_s;                /* worker wall time spent stepping */
    int64_t device_bytes;         /* now */
    int64_t peak_device_bytes;    /* highest after an admission */
} pic_server_stats_t;

/* common: grid resolution, cfl, wavelength, sort interval, device, budget (as
 * pic_batch_create).  max_runs: batch slots.  chunk_steps (>= 1, rounded up to
 * a multiple of the sort interval): steps between admission points. */
pic_status pic_server_create(const pic_config* common, int max_runs, int64_t chunk_steps, pic_server** out);
/* Queue a run.  Its results: the ion and electron spectra dN/dE over nbins
 * equal bins of [0, ion_e_max_MeV) and [0, el_e_max_MeV), and the energy
 * read-out of pic_energy, all at the run's last step.  *ticket identifies the
 * request.  PIC_ERR_OOM if the run alone exceeds the budget;
 * PIC_ERR_INVALID_ARG for an invalid description (checked as
 * pic_batch_add_run checks it, at admission: the request then fails). */
pic_status pic_server_submit(pic_server* srv, const pic_run_desc* desc, int nbins, double ion_e_max_MeV,
                             double el_e_max_MeV, int64_t* ticket);
/* Wait up to wait_s seconds (0: do not wait) for a request.  PIC_OK: the
 * outputs (caller-owned ion_counts[nbins], el_counts[nbins], energy[6]; each
 * nullable) and *latency_s (submission to result) are written and the ticket
 * is forgotten.  PIC_ERR_TIMEOUT: not finished yet.  A request that failed
 * returns its error (and is forgotten).  PIC_ERR_INVALID_ARG: unknown ticket. */
pic_status pic_server_result(pic_server* srv, int64_t ticket, double wait_s, double* ion_counts, double* el_counts,
                             double* energy, double* latency_s);
/* Admission policy: PIC_SERVE_FIFO (arrival order, the default) or
 * PIC_SERVE_SHORTEST_FIRST (least particles x steps first, ties in arrival
 * order); max_resident_particles (0: no cap) bounds the particles stepping
 * at once, so that admitted runs are not slowed by an ever larger batch
 * (a request is always admitted when nothing is running). */
enum { PIC_SERVE_FIFO = 0, PIC_SERVE_SHORTEST_FIRST = 1 };
pic_status pic_server_set_policy(pic_server* srv, int policy, int64_t max_resident_particles);
pic_status pic_server_stats(pic_server* srv, pic_server_stats_t* out);
/* Cancel a request: a queued one is dropped at once; a running one leaves the
 * batch at the end of the current step chunk and its memory is freed.  Its
 * result then reports PIC_ERR_STATE ("cancelled").  PIC_ERR_STATE if it has
 * already finished; PIC_ERR_INVALID_ARG for an unknown ticket. */
pic_status pic_server_cancel(pic_server* srv, int64_t ticket);
/* Message of the last failed server call of the calling thread. */
const char* pic_server_last_error(const pic_server* srv);
/* Stop the worker (unfinished requests are dropped) and free everything. */
pic_status pic_server_destroy(pic_server* srv);

/* ---- Single electrons in analytic plane waves (the paper's validation path) --
 * Integrates many independent electrons (charge -1) at once, one GPU thread
 * each, in double precision: a reference integrator for scans over
 * amplitude and initial momentum, as in Sec. 3 (the paper's single-particle
 * test against the lab-frame LL equation), not the PIC step.
 * Plane waves travel along +x with phase phi = t - x and B = x_hat x E:
 *   wave 0: LP, Ey = a0 cos(phi);
 *   wave 1: CP, (Ey, Ez) = (a0/sqrt2) (cos(phi), sin(phi));
 *   wave 2: LP pulse, Ey = a0 sin^2(pi phi/tau) cos(phi) for 0 <= phi <= tau, else 0.
 * Integrators: PIC_INTEGRATOR_LEAPFROG, the pusher of Sec. 3 (Boris + the RR
 * kick of Eqs. f_r, pertfull, estim1, estimgamma; initial data x(0) = x0 and
 * p^{-1/2} = p0; rows hold t_{n+1}, x^{n+1}, p^{n+1/2}); PIC_INTEGRATOR_RK4,
 * classical RK4 on Eq. (3dLL) (x(0) = x0, p(0) = p0; rows hold t, x, p at the
 * same time).  flags: PIC_ELECTRON_RR adds radiation reaction (eps from
 * lambda_um); PIC_ELECTRON_DERIV keeps the field-derivative term of
 * Eq. (3dLL) (RK4 only).  out: caller-owned host array [n][nsamples][5], row k
 * of case c taken after (k+1)*every steps (nsamples <= nsteps/every).
 * Synchronous. */
typedef struct {
    int wave;        /* 0, 1 or 2 as above */
    double a0, tau;  /* amplitude; pulse length in 1/omega (wave 2) */
    double x0;       /* initial position, c/omega */
    double p0[3];    /* initial momentum, m c */
} pic_electron_case;
enum { PIC_INTEGRATOR_LEAPFROG = 0, PIC_INTEGRATOR_RK4 = 1 };
enum { PIC_ELECTRON_RR = 1, PIC_ELECTRON_DERIV = 2 };
pic_status pic_electron_scan(const pic_electron_case* cases, int64_t n, int integrator, int flags, double dt,
                             int64_t nsteps, int every, double lambda_um, int device, double* out,
                             int64_t nsamples);

/* ---- Spectrum without device allocation -----------------------------------
 * The paper has no counterpart to this entry point; it exists for callers of
 * this library that cannot allocate device memory when they need a spectrum:
 * code that must not synchronise the GPU (cudaMalloc and cudaFree can), code
 * whose device memory is owned by another allocator under a fixed budget, or
 * a plugin that is handed device buffers by its host application.
 *
 * It computes what pic_spectra computes for one species, from momenta the
 * caller already holds on the device, and allocates nothing: its integer bin
 * counters live in one fixed array inside the library, sized for
 * PIC_NOALLOC_MAX_BINS bins (plus under- and overflow, 8 bytes each, about
 * 0.5 MB), which every GPU that loads the library keeps until the process
 * exits.
 *
 *   px, py, pz   device arrays of n floats, momenta in m_s c (caller-owned)
 *   mass_me      particle mass in electron masses (E = m c^2 (gamma - 1))
 *   weight_dx    weight * dx of one macro-particle (the count unit)
 *   counts       device array of nbins doubles (caller-owned), receives
 *                weight_dx * (particles in bin k) / bin width, as pic_spectra
 *   stream       cudaStream_t to run on (NULL: the legacy default stream)
 *
 * Runs on the current device, asynchronously on `stream`; the result is ready
 * when the stream reaches it.  nbins outside [1, PIC_NOALLOC_MAX_BINS] is
 * rejected with PIC_ERR_INVALID_ARG; pic_last_error(NULL) gives the reason.
 * The first call on a device looks up the counter array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the counter array: each call
 * clears it before counting, so calls in sequence are independent, but calls
 * whose work overlaps on the GPU (other streams or threads) race on it. */
#define PIC_NOALLOC_MAX_BINS 65536
pic_status pic_spectrum_noalloc(const float* px, const float* py, const float* pz, int64_t n,
                                double mass_me, double weight_dx, int nbins, double e_min_MeV,
                                double e_max_MeV, double* counts, void* stream);

#ifdef __cplusplus
}
#endif
#endif
