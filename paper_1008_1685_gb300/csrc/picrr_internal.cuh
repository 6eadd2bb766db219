// Internal layout, constants and device helpers of the picrr CUDA library.
//
// A batch holds R independent runs (a single simulation handle is a batch of
// one).  The kernels of one step process all active runs of the batch in one
// launch each; a device table of RunDev entries gives every run's arrays and
// parameters.
//
// Data layout in HBM (per run):
//   grid arrays   float, Nx+1+2*PADF elements (rounded up to 4), element
//                 PADF holds node / half node 0; the guard elements are zero.
//                 Ex, Ey, Ez, By, Bz are ping-ponged by the Yee kernel.
//   accumulators  int64 fixed point (2^fp units) for Jx (half nodes) and
//                 Jy, Jz (nodes), two sets alternating by step parity; the
//                 set of the last step holds its current until the next
//                 step's Yee update zeroes it (read-back converts it).
//   particles     per species, structure of arrays, two buffers each
//                 (ping-ponged by the sort): cell int32, off/px/py/pz float,
//                 id int32.  A particle that left the box is frozen at the
//                 wall and stored with cell = -1 - k, k its last cell (0 at
//                 x = 0, Nx-1 at x = L); it keeps sorting under k.
// Per batch:
//   units         work units of at most UNIT_P consecutive particles of one
//                 run and species whose cells at the last sort lie in one
//                 tile of TILE cells.
#pragma once

#include <cuda_runtime.h>

#include "picrr.h"
#include <stdint.h>

namespace picrr {

constexpr int PADF = 40;          // guard elements left of index 0 of every grid array
constexpr int TILE = 64;          // cells per tile: a dense tile is split into units of at most unit_p particles
// Consecutive tiles that form one unit when they hold <= unit_p particles (else each aligned half
// group that does; else single tiles).  Groups of 8 instead of 4 took thinly spread plasma's push
// from 0.651 to 0.595 ms (fewer, longer units) and the 256-run scan's late phase from 0.569 to 0.551.
constexpr int GROUP = 8;
constexpr int SPAN = GROUP * TILE;  // cell span bound of a unit
constexpr int UNIT_P = 4096;      // default particles per unit at most (unit_p, a run-time shape of a batch)
constexpr int UNIT_P_MIN = 1024;  // smallest unit_p (the bound used for memory estimates)
constexpr int UNIT_P_MAX = 16384;
// Largest sort interval.  The push barely slows with the steps since the sort (+0.2 % from the first to
// the last 8 steps of a 64-step interval), so longer intervals amortise the sort: 96 keeps the push
// kernel's shared memory static (46 KB with 4 particles per thread); 128 needs dynamic shared memory,
// with which the same kernel ran 1.5 % (dense) to 2.8 % (thin) slower.
constexpr int KMAX = 96;
constexpr int PUSH_T = 256;       // threads of the push kernel
constexpr int WMAX = SPAN + 2 * KMAX + 16;  // window length bound in the push kernel (>= SPAN + 2 KMAX + 9)
constexpr int SSTR = SPAN + 2 * KMAX + 4;   // per-unit key-window stride of the sort scratch (>= SPAN + 2 KMAX)
constexpr int FIELD_T = 128;      // threads of the Yee kernel
// Nodes per thread of the Yee kernel.  Measured per step (1 / 2 / 4 / 8): 256 runs of 15,000
// cells 0.082 / 0.075 / 0.073 / 0.081 ms, one run of 200,000 cells 0.0102 / 0.0107 / 0.0121 /
// 0.0144 ms (too few blocks for the SMs at 4 and 8); one node per thread with the current
// staged through shared memory and the last loads issued after the barriers took 0.096 ms.
#ifndef PICRR_FIELD_NPT
#define PICRR_FIELD_NPT 2
#endif
constexpr int FIELD_NODES = FIELD_T * PICRR_FIELD_NPT;  // nodes per block of the Yee kernel
constexpr int KEY_T = 256;        // cells per block of the per-cell sort kernels
constexpr int WAIT_LIMIT = 1 << 22;  // bounded spin on an mbarrier before reporting a timeout

// Device status bits (pic_step_n reads them after each call).
constexpr int ST_TIMEOUT = 1;
constexpr int ST_WINDOW = 2;      // a particle left its unit window (cannot happen when cfl < 1)

struct DevSpecies {
    int32_t* cell;
    float* off;
    float* px;
    float* py;
    float* pz;
    int32_t* id;
};

struct UnitTable {
    int32_t* run;      // [max_units] run of the unit
    int32_t* species;  // species of the unit
    int32_t* start;    // first particle index (in the run's arrays)
    int32_t* end;      // one past the last
    int32_t* lo;       // cell of the first particle at the last sort
    int32_t* hi;       // cell of the last particle at the last sort
    int32_t* count;    // [1]: total units
};

// One run of a batch, as the kernels see it.
struct RunDev {
    DevSpecies sp[2][2];   // [species][particle buffer]
    int32_t n[2];          // particles per species
    float qm[2];           // charge / mass
    float qw[2];           // charge * weight
    float rad_w[2];        // weight * dx * mass (energy per unit gamma)
    float lscale[2];       // 32-bit fixed-point scale of a warp deposit record (power of two)
    int32_t lshift[2];     // shift from warp records to accumulator units
    int32_t rr;            // radiation reaction on electrons
    int32_t active;        // stepped by the batch
    int32_t Nx, is, glen;
    int32_t fpar;          // field / current buffer at batch step g: (g + fpar) & 1
    float fp_inv;          // 2^-fp of the current accumulators
    float* F[2][5];        // [buffer][Ex, Ey, Ez, By, Bz], padded
    unsigned long long* J[2][3];  // [parity][Jx, Jy, Jz], padded
    double* tally;         // [4]: radiated, flux in, flux out, spare
    int32_t* keycount[2];  // sort scratch per species: [Nx + 2]
    int32_t* keystart[2];  // [Nx + 2]; keystart[Nx] = particles
    int32_t* blocksum[2];  // [Nx / 256 + 2]
    int32_t* blockstart[2];
    int32_t* tile_n[2];    // [Nx / TILE + 3]
    int32_t* tile_first[2];
};

struct PushParams {
    const RunDev* runs;
    UnitTable units;
    double* rad_part;   // [max_units] radiated energy of each unit since the last flush
    int* status;
    int64_t gstep;      // batch step
    int k;              // steps since the last sort
    int cur;            // particle buffer
    float cfl, dt, eps;
};

struct LaserParams {
    int on, pol, env;
    double a0, tau, rise;
};

struct FieldParams {
    const RunDev* runs;
    const int32_t* blk_run;  // [blocks] run of each block
    const int32_t* blk_i0;   // [blocks] first node of each block
    // per run: incident field (ay, az) at retarded times t_n (source node),
    // t_n + dt/2 + dx/2 (half node before it) and t_{n+1}:
    // Ey_inc = Bz_inc = ay, Ez_inc = -By_inc = az
    const float* inc;        // [runs * 6]
    int64_t gstep;
    double dt;
    float c, hc, fdt;        // cfl, cfl/2, dt
};

// ---------------------------------------------------------------------------
// PTX helpers: mbarrier and the bulk (non-tensor) TMA copy global -> shared.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait: returns false after WAIT_LIMIT polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (int it = 0; it < WAIT_LIMIT; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// 1D bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
// from global to this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_1d(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// Host-side launch wrappers (each defined in its own translation unit).
// ---------------------------------------------------------------------------
void launch_push(const PushParams& P, int grid, int slot_w, cudaStream_t st);  // slot_w: 4 or 2 particles per thread and round
void launch_field(const FieldParams& P, int grid, cudaStream_t st);

struct SortParams {
    RunDev* runs;
    int nruns;
    UnitTable units;
    int32_t* cnt;          // [max_units * SSTR] key counts per unit window
    int32_t* offs;         // [max_units * SSTR] destinations per unit window
    int32_t* rs_units;     // [4 * nruns]: units per (run, species) pair, then the first unit of each pair
    int* status;
    int k, cur, max_units;
    int kb_max;            // key blocks of the largest run: ceil(max Nx / 256)
    int unit_p;            // particles per unit at most (UNIT_P_MIN..UNIT_P_MAX)
};
// Full re-sort of every active run (bounded displacement since the last sort)
// and the new unit table; particles move from buffer cur to 1 - cur.
void launch_sort(const SortParams& S, cudaStream_t st, int* launches);
// Unit table of every active run from its current, already sorted particles.
void launch_build_units(const SortParams& S, cudaStream_t st, int* launches);
// Add each run's per-unit radiated energy into its tally[0]; zero them.
// rs_units as in SortParams.
void launch_rad_flush(const RunDev* runs, int nruns, const int32_t* rs_units, double* rad_part, cudaStream_t st);

void launch_foil(DevSpecies e, DevSpecies ion, int c0, int ncell, int ppc, uint64_t seed, cudaStream_t st);
void launch_iota(int32_t* id, int64_t n, cudaStream_t st);
}  // namespace picrr
#include <string>
namespace picrr {
// record the message returned by pic_last_error(NULL) on this thread
void set_null_handle_error(const std::string& msg);

// Diagnostics.
struct DiagParams {
    const float* F[5];
    int Nx, is;
    float hc;
};
// Writes double out_partials[grid]; returns grid used.
int launch_field_energy(const DiagParams& D, double* partials, int max_blocks, cudaStream_t st);
int launch_kinetic(DevSpecies sp, int64_t n, double* partials, int max_blocks, cudaStream_t st);
void launch_reduce_partials(const double* partials, int n, double scale, double* out, cudaStream_t st);
void launch_spectrum(DevSpecies sp, int64_t n, double mass_mev, int nbins, double e_min, double e_max,
                     unsigned long long* bins, cudaStream_t st);

// Friction coefficient d (Eq. damping) and quantum parameter chi per particle
// from the stored momentum and the fields at the particle.  d_out / chi_out
// (nullable) in stored order; out[0], out[1]: float bits of max d and max chi
// (atomicMax on the bits of non-negative floats); out[2]: count of chi >= chi_flag.
struct SnapParams {
    const float* F[5];
    float eps, ecr_inv, chi_flag;
};
void launch_wait_selftest(int* status, cudaStream_t st);
void launch_validate(const int32_t* cell, const float* off, const float* px, const float* py, const float* pz,
                     int64_t n, int Nx, unsigned long long* out, cudaStream_t st);
void launch_electron_scan(const pic_electron_case* cases, int64_t n, int integrator, int flags, double dt,
                          int64_t nsteps, int every, double eps, double* out, int64_t nsamples, cudaStream_t st);

void launch_snapshot(DevSpecies sp, int64_t n, const SnapParams& S, float* d_out, float* chi_out,
                     unsigned long long* out, cudaStream_t st);

}  // namespace picrr
