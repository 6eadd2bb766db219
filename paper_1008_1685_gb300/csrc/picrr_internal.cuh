// Internal layout, constants and device helpers of the picrr CUDA library.
//
// Data layout in HBM (one handle):
//   grid arrays   float, Nx+1+2*PADF elements (rounded up to 4), element
//                 PADF holds node / half node 0; the guard elements are zero.
//                 Ex, Ey, Ez, By, Bz are ping-ponged by the Yee kernel.
//   accumulators  int64 fixed point (2^fp units) for Jx (half nodes) and
//                 Jy, Jz (nodes), two sets alternating by step parity.
//   particles     per species, structure of arrays, two buffers each
//                 (ping-ponged by the sort): cell int32, off/px/py/pz float,
//                 id int32.  cell < 0 marks a particle frozen at a wall
//                 (-1: x = 0, -2: x = L).
//   units         work units of at most UNIT_P consecutive particles whose
//                 cells at the last sort lie in one tile of TILE cells.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace picrr {

constexpr int PADF = 40;          // guard elements left of index 0 of every grid array
constexpr int TILE = 64;          // cells per tile: bounds the cell span of a unit
constexpr int UNIT_P = 2048;      // particles per unit at most
constexpr int KMAX = 32;          // largest sort interval
constexpr int PUSH_T = 256;       // threads of the push kernel
constexpr int WMAX = 144;         // window length bound in the push kernel (>= TILE + 2 KMAX + 10)
constexpr int SSTR = TILE + 2 * KMAX + 4;  // per-unit key-window stride of the sort scratch
constexpr int FIELD_T = 256;      // nodes per block of the Yee kernel
constexpr int NQ = 5;             // deposit quantities per bin: jy_lo, jy_hi, jz_lo, jz_hi, jx
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
    int32_t* species;  // [max_units]
    int32_t* start;    // first particle index
    int32_t* end;      // one past the last
    int32_t* lo;       // cell of the first particle at the last sort
    int32_t* hi;       // cell of the last particle at the last sort
    int32_t* count;    // [3]: total units, units of species 0, units of species 1
};

struct PushParams {
    DevSpecies sp[2];
    float qm[2];        // charge / mass
    float qw[2];        // charge * weight
    float rad_w[2];     // weight * dx * mass (energy per unit gamma)
    int rr[2];          // radiation reaction on this species
    const float* F[5];  // Ex, Ey, Ez, By, Bz, each pointing at element 0 of the padded array
    unsigned long long* J[3];  // Jx, Jy, Jz accumulators (padded)
    UnitTable units;
    double* rad_part;   // [max_units] radiated energy of each unit since the last flush
    int* status;
    int Nx;
    int k;              // steps since the last sort
    float cfl, dt, eps;
    float lscale[2];    // per-species 32-bit fixed-point scale of a warp record (power of two)
    int lshift[2];      // fp - log2(lscale): shift from warp records to accumulator units
};

struct LaserParams {
    int on, pol, env;
    double a0, tau, rise;
};

struct FieldParams {
    const float* Fo[5];  // fields at time n (padded)
    float* Fn[5];        // fields at time n+1 (padded)
    const unsigned long long* Jacc[3];  // this step's accumulators
    unsigned long long* Jnext[3];       // zeroed for the next step
    float* Jf[3];        // float J of this step (read-back)
    double* tally;       // [0] radiated, [1] flux in, [2] flux out
    int Nx, is;
    int glen;            // length of every padded grid array
    int64_t n;           // step index (t_n = n dt)
    double dt, dx;
    float c, hc, fdt;    // cfl, cfl/2, dt
    float fp_inv;        // 2^-fp
    // incident field (ay, az) at retarded times t_n (source node), t_n + dt/2 + dx/2
    // (half node before it) and t_{n+1}: Ey_inc = Bz_inc = ay, Ez_inc = -By_inc = az
    float inc[6];
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
void launch_push(const PushParams& P, int grid, cudaStream_t st);
void launch_field(const FieldParams& P, int grid, cudaStream_t st);

struct SortParams {
    DevSpecies src[2], dst[2];
    int64_t n[2];          // particle count per species
    UnitTable units;
    int32_t* cnt;          // [max_units * SSTR] key counts per unit window
    int32_t* offs;         // [max_units * SSTR] destinations per unit window
    int32_t* esc_cnt;      // [max_units]
    int32_t* esc_off;      // [max_units]
    int32_t* keycount[2];  // [Nx + 2]
    int32_t* keystart[2];  // [Nx + 2]; keystart[Nx] = active count
    int32_t* meta;         // [8]: [0..1] active particles at the last sort, [2..3] escapes since,
                           // [4] error bits of the sort
    int32_t* blocksum[2];  // [Nx/256 + 1] key counts per block of 256 cells
    int32_t* blockstart[2];
    int32_t* tile_n[2];    // [Nx/TILE + 1] units per tile
    int32_t* tile_first[2];  // [Nx/TILE + 2] first unit of each tile
    int Nx, k, max_units;
};
// Full re-sort of both species (bounded displacement since the last sort).
void launch_sort(const SortParams& S, int n_unit_blocks, cudaStream_t st, int* launches);
// Unit table from already sorted particles (after loading).
void launch_build_units_from_sorted(const SortParams& S, cudaStream_t st, int* launches);

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
// tally[0] += sum of rad_part[0 .. units.count[0]) in a fixed order; zero them.
void launch_rad_flush(double* rad_part, const int32_t* unit_count, double* tally, cudaStream_t st);
void launch_spectrum(DevSpecies sp, int64_t n, double mass_mev, int nbins, double e_min, double e_max,
                     unsigned long long* bins, cudaStream_t st);

}  // namespace picrr
