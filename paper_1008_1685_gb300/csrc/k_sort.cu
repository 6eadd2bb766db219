// Periodic cell sort of the particles and the unit table built from it.
//
// The sort is a stable counting sort by cell (particles frozen at a wall go
// last, in their previous order).  It exploits what the push guarantees:
// a particle moves less than one cell per step, so k steps after the last
// sort every particle of unit u has a cell in [lo_u - k, hi_u + k].  Hence
//   1. each unit counts its particles per cell of that window (shared-memory
//      integer atomics);
//   2. for each cell the units whose window covers it form a contiguous
//      range (lo and hi are sorted), found by binary search; the per-cell
//      totals are scanned into the new cell starts, and every (unit, cell)
//      pair gets its destination offset in unit order;
//   3. each unit scatters its particles, ranking equal cells in index order
//      (warp match + per-warp counts combined in warp order), so the result
//      does not depend on scheduling;
//   4. the unit table is rebuilt from the sorted cells: tiles of TILE cells,
//      split into chunks of at most UNIT_P particles.
// Every particle is read once and written once; the cell array is read
// once more for the counts.
#include <algorithm>

#include "picrr_internal.cuh"

namespace picrr {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int SORT_T = 256;
constexpr int SCAN_T = 1024;
constexpr int ESC = SSTR - 1;  // local slot of particles frozen since the last sort

__device__ __forceinline__ int unit_base(const UnitTable& U, int s) { return s == 0 ? 0 : U.count[1]; }

// ---- 1. per-unit window counts -------------------------------------------
__global__ void __launch_bounds__(SORT_T) k_sort_count(const SortParams S) {
    __shared__ int cnt[SSTR];
    const int u = blockIdx.x;
    if (u >= S.units.count[0]) return;
    const int s = S.units.species[u];
    const int start = S.units.start[u], end = S.units.end[u];
    const int wb = S.units.lo[u] - S.k;
    const int L = S.units.hi[u] + S.k + 1 - wb;
    for (int i = threadIdx.x; i < SSTR; i += SORT_T) cnt[i] = 0;
    __syncthreads();
    const int32_t* cell = S.src[s].cell;
    for (int i = start + threadIdx.x; i < end; i += SORT_T) {
        const int c = cell[i];
        if (c < 0) {
            atomicAdd(&cnt[ESC], 1);
        } else {
            const int l = c - wb;
            if (l >= 0 && l < L && l < ESC) atomicAdd(&cnt[l], 1);
            else atomicOr(S.meta + 4, ST_WINDOW);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SSTR; i += SORT_T) S.cnt[static_cast<size_t>(u) * SSTR + i] = (i == ESC) ? 0 : cnt[i];
    if (threadIdx.x == 0) S.esc_cnt[u] = cnt[ESC];
}

// Units of species s covering cell key: [u0, u1] (empty if u0 > u1).
__device__ void covering(const SortParams& S, int s, int key, int& u0, int& u1) {
    const int b = unit_base(S.units, s), n = S.units.count[1 + s];
    // first u with hi + k >= key
    int l = 0, r = n;
    while (l < r) {
        const int m = (l + r) >> 1;
        if (S.units.hi[b + m] + S.k >= key) r = m; else l = m + 1;
    }
    u0 = b + l;
    // last u with lo - k <= key
    l = 0;
    r = n;
    while (l < r) {
        const int m = (l + r) >> 1;
        if (S.units.lo[b + m] - S.k <= key) l = m + 1; else r = m;
    }
    u1 = b + l - 1;
}

// ---- 2a. per-cell totals ----------------------------------------------------
__global__ void k_sort_totals(const SortParams S) {
    const int s = blockIdx.y;
    const int key = blockIdx.x * blockDim.x + threadIdx.x;
    if (key >= S.Nx) return;
    int u0, u1;
    covering(S, s, key, u0, u1);
    int tot = 0;
    for (int u = u0; u <= u1; ++u) {
        const int l = key - (S.units.lo[u] - S.k);
        if (l >= 0 && l < ESC) tot += S.cnt[static_cast<size_t>(u) * SSTR + l];
    }
    S.keycount[s][key] = tot;
}

// ---- 2b. exclusive scan of the cell totals (one block per species) --------
// keystart[s][0..Nx], keystart[Nx] = active count.  Also the escape offsets
// of the units (after the active particles) and meta[2+s] = new escapes.
__global__ void __launch_bounds__(SCAN_T) k_sort_scan(const SortParams S, int with_units) {
    __shared__ int warp_tot[SCAN_T / 32];
    __shared__ int carry;
    const int s = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = S.Nx;
    const int per = (n + SCAN_T - 1) / SCAN_T;
    const int a = min(n, tid * per), b = min(n, a + per);
    int sum = 0;
    for (int i = a; i < b; ++i) sum += S.keycount[s][i];
    // block exclusive scan of the per-thread sums
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        warp_tot[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    int run = x - sum + (warp > 0 ? warp_tot[warp - 1] : 0);
    for (int i = a; i < b; ++i) {
        S.keystart[s][i] = run;
        run += S.keycount[s][i];
    }
    if (tid == SCAN_T - 1) {
        S.keystart[s][n] = warp_tot[SCAN_T / 32 - 1];
        carry = warp_tot[SCAN_T / 32 - 1];
    }
    if (!with_units) return;
    __syncthreads();
    // escape offsets of the units of species s, in unit order
    const int ub = unit_base(S.units, s), nu = S.units.count[1 + s];
    const int act = carry;
    __syncthreads();
    int base = 0;
    for (int c0 = 0; c0 < nu; c0 += SCAN_T) {
        const int u = c0 + tid;
        const int v = (u < nu) ? S.esc_cnt[ub + u] : 0;
        int y = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int z = __shfl_up_sync(FULL, y, o);
            if (lane >= o) y += z;
        }
        __syncthreads();
        if (lane == 31) warp_tot[warp] = y;
        __syncthreads();
        if (warp == 0) {
            int w = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int z = __shfl_up_sync(FULL, w, o);
                if (lane >= o) w += z;
            }
            warp_tot[lane] = w;
        }
        __syncthreads();
        const int excl = base + y - v + (warp > 0 ? warp_tot[warp - 1] : 0);
        if (u < nu) S.esc_off[ub + u] = act + excl;
        base += warp_tot[SCAN_T / 32 - 1];
    }
    if (tid == 0) S.meta[2 + s] = base;
}

// ---- 2c. destination of every (unit, cell) pair ---------------------------
__global__ void k_sort_offsets(const SortParams S) {
    const int s = blockIdx.y;
    const int key = blockIdx.x * blockDim.x + threadIdx.x;
    if (key >= S.Nx) return;
    int u0, u1;
    covering(S, s, key, u0, u1);
    int run = S.keystart[s][key];
    for (int u = u0; u <= u1; ++u) {
        const int l = key - (S.units.lo[u] - S.k);
        if (l >= 0 && l < ESC) {
            const size_t q = static_cast<size_t>(u) * SSTR + l;
            S.offs[q] = run;
            run += S.cnt[q];
        }
    }
}

__device__ __forceinline__ void copy_particle(const DevSpecies& a, DevSpecies& b, int i, int d) {
    b.cell[d] = a.cell[i];
    b.off[d] = a.off[i];
    b.px[d] = a.px[i];
    b.py[d] = a.py[i];
    b.pz[d] = a.pz[i];
    b.id[d] = a.id[i];
}

// ---- 3. stable scatter ------------------------------------------------------
__global__ void __launch_bounds__(SORT_T) k_sort_scatter(const SortParams S) {
    __shared__ int base[SSTR];
    __shared__ int wcnt[SORT_T / 32][SSTR];
    const int u = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (u >= S.max_units) {
        // particles frozen before the last sort keep their order at the very end
        for (int s = 0; s < 2; ++s) {
            const int old_act = S.meta[s];
            const int dst0 = S.keystart[s][S.Nx] + S.meta[2 + s];
            DevSpecies dst = S.dst[s];
            for (int i = old_act + (u - S.max_units) * SORT_T + tid; i < S.n[s];
                 i += (gridDim.x - S.max_units) * SORT_T)
                copy_particle(S.src[s], dst, i, dst0 + (i - old_act));
        }
        return;
    }
    if (u >= S.units.count[0]) return;
    const int s = S.units.species[u];
    const int start = S.units.start[u], end = S.units.end[u];
    const int wb = S.units.lo[u] - S.k;
    const DevSpecies src = S.src[s];
    DevSpecies dst = S.dst[s];
    for (int i = tid; i < SSTR; i += SORT_T) base[i] = 0;
    for (int i = tid; i < (SORT_T / 32) * SSTR; i += SORT_T) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int c0 = start; c0 < end; c0 += SORT_T) {
        const int i = c0 + tid;
        int key = -1;
        if (i < end) {
            const int c = src.cell[i];
            if (c < 0) key = ESC;
            else {
                const int l = c - wb;
                key = (l >= 0 && l < ESC) ? l : -1;  // out of window cannot happen (counted as error)
            }
        }
        const unsigned peers = __match_any_sync(FULL, key);
        const int rw = __popc(peers & lt);
        const bool leader = (__ffs(peers) - 1) == lane;
        if (leader && key >= 0) wcnt[warp][key] = __popc(peers);
        __syncthreads();
        int dest = -1;
        if (key >= 0) {
            int r = base[key] + rw;
            for (int w = 0; w < warp; ++w) r += wcnt[w][key];
            dest = (key == ESC) ? S.esc_off[u] + r : S.offs[static_cast<size_t>(u) * SSTR + key] + r;
        }
        __syncthreads();
        if (leader && key >= 0) {
            atomicAdd(&base[key], __popc(peers));
            wcnt[warp][key] = 0;
        }
        __syncthreads();
        if (dest >= 0) copy_particle(src, dst, i, dest);
    }
}

// ---- 4. unit table from sorted cells (one block, both species) -------------
__global__ void __launch_bounds__(SCAN_T) k_build_units(const SortParams S) {
    __shared__ int warp_tot[SCAN_T / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ntiles = (S.Nx + TILE - 1) / TILE;
    int ubase = 0;
    for (int s = 0; s < 2; ++s) {
        const int32_t* ks = S.keystart[s];
        const int32_t* cell = S.dst[s].cell;
        int run = 0;
        for (int t0 = 0; t0 < ntiles; t0 += SCAN_T) {
            const int t = t0 + tid;
            int nt = 0, ts = 0, te = 0;
            if (t < ntiles) {
                ts = ks[t * TILE];
                te = ks[min((t + 1) * TILE, S.Nx)];
                nt = (te - ts + UNIT_P - 1) / UNIT_P;
            }
            int y = nt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int z = __shfl_up_sync(FULL, y, o);
                if (lane >= o) y += z;
            }
            __syncthreads();
            if (lane == 31) warp_tot[warp] = y;
            __syncthreads();
            if (warp == 0) {
                int w = warp_tot[lane];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int z = __shfl_up_sync(FULL, w, o);
                    if (lane >= o) w += z;
                }
                warp_tot[lane] = w;
            }
            __syncthreads();
            const int first = ubase + run + y - nt + (warp > 0 ? warp_tot[warp - 1] : 0);
            for (int r = 0; r < nt; ++r) {
                const int u = first + r;
                if (u >= S.max_units) break;  // cannot happen: max_units bounds the count
                const int a = ts + r * UNIT_P, b = min(a + UNIT_P, te);
                S.units.species[u] = s;
                S.units.start[u] = a;
                S.units.end[u] = b;
                S.units.lo[u] = cell[a];
                S.units.hi[u] = cell[b - 1];
            }
            run += warp_tot[SCAN_T / 32 - 1];
        }
        if (tid == 0) {
            S.units.count[1 + s] = run;
            S.meta[s] = ks[S.Nx];  // active particles at this sort
        }
        ubase += run;
        __syncthreads();
    }
    if (tid == 0) S.units.count[0] = min(ubase, S.max_units);
}

// ---- histogram of sorted, freshly loaded particles ---------------------------
__global__ void k_hist(const SortParams S) {
    const int s = blockIdx.y;
    const int64_t n = S.n[s];
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int c = S.dst[s].cell[i];
        if (c >= 0 && c < S.Nx) atomicAdd(&S.keycount[s][c], 1);
    }
}

}  // namespace

void launch_sort(const SortParams& S, int n_unit_blocks, cudaStream_t st, int* launches) {
    const int kb = (S.Nx + 255) / 256;
    k_sort_count<<<n_unit_blocks, SORT_T, 0, st>>>(S);
    k_sort_totals<<<dim3(kb, 2), 256, 0, st>>>(S);
    k_sort_scan<<<2, SCAN_T, 0, st>>>(S, 1);
    k_sort_offsets<<<dim3(kb, 2), 256, 0, st>>>(S);
    k_sort_scatter<<<n_unit_blocks + 64, SORT_T, 0, st>>>(S);
    k_build_units<<<1, SCAN_T, 0, st>>>(S);
    *launches += 6;
}

void launch_build_units_from_sorted(const SortParams& S, cudaStream_t st, int* launches) {
    cudaMemsetAsync(S.keycount[0], 0, sizeof(int32_t) * (S.Nx + 2), st);
    cudaMemsetAsync(S.keycount[1], 0, sizeof(int32_t) * (S.Nx + 2), st);
    k_hist<<<dim3(256, 2), 256, 0, st>>>(S);
    k_sort_scan<<<2, SCAN_T, 0, st>>>(S, 0);
    k_build_units<<<1, SCAN_T, 0, st>>>(S);
    *launches += 3;
}

// ---- foil loader -------------------------------------------------------------
namespace {
// SplitMix64 (Steele, Lea and Flood 2014): n-th output from state `seed`.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t n) {
    uint64_t z = seed + n * 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void k_foil(DevSpecies e, DevSpecies ion, int c0, int ncell, int ppc, uint64_t seed) {
    const int64_t n = static_cast<int64_t>(ncell) * ppc;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int c = c0 + static_cast<int>(i / ppc);
        const int kk = static_cast<int>(i % ppc);
        const uint64_t r = splitmix64_at(seed, static_cast<uint64_t>(c) * static_cast<uint64_t>(ppc) +
                                                   static_cast<uint64_t>(kk) + 1ull);
        const float off = static_cast<float>(r >> 40) * (1.0f / 16777216.0f);  // exact: 24-bit dyadic
        e.cell[i] = c;
        ion.cell[i] = c;
        e.off[i] = off;
        ion.off[i] = off;
        e.px[i] = e.py[i] = e.pz[i] = 0.f;
        ion.px[i] = ion.py[i] = ion.pz[i] = 0.f;
        e.id[i] = static_cast<int32_t>(i);
        ion.id[i] = static_cast<int32_t>(i);
    }
}
}  // namespace

namespace {
__global__ void k_iota(int32_t* id, int64_t n) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        id[i] = static_cast<int32_t>(i);
}
}  // namespace

void launch_iota(int32_t* id, int64_t n, cudaStream_t st) {
    const int grid = static_cast<int>(std::min<int64_t>((n + 255) / 256, 152 * 64));
    k_iota<<<grid > 0 ? grid : 1, 256, 0, st>>>(id, n);
}

void launch_foil(DevSpecies e, DevSpecies ion, int c0, int ncell, int ppc, uint64_t seed, cudaStream_t st) {
    const int64_t n = static_cast<int64_t>(ncell) * ppc;
    const int grid = static_cast<int>(std::min<int64_t>((n + 255) / 256, 152 * 64));
    k_foil<<<grid > 0 ? grid : 1, 256, 0, st>>>(e, ion, c0, ncell, ppc, seed);
}

}  // namespace picrr
