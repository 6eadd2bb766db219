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
constexpr int KEY_T = 256;  // keys per block of the per-cell kernels
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
    const int lane = threadIdx.x & 31;
    for (int i0 = start; i0 < end; i0 += SORT_T) {  // block-uniform trip count
        const int i = i0 + threadIdx.x;
        int l = -1;
        if (i < end) {
            const int c = cell[i];
            if (c < 0) {
                l = ESC;
            } else {
                l = c - wb;
                if (!(l >= 0 && l < L && l < ESC)) {
                    atomicOr(S.meta + 4, ST_WINDOW);
                    l = -1;
                }
            }
        }
        // lanes with the same cell add their count once
        const unsigned peers = __match_any_sync(FULL, l);
        if (l >= 0 && lane == __ffs(peers) - 1) atomicAdd(&cnt[l], __popc(peers));
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

__device__ __forceinline__ int block_sum_int(int v, int* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    int t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < KEY_T / 32; ++w) t += sh[w];
    return t;
}

// exclusive scan of v over the block (KEY_T threads), plus the block total
__device__ __forceinline__ int block_excl_scan(int v, int* sh, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < KEY_T / 32 ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        if (lane < KEY_T / 32) sh[lane] = w;
    }
    __syncthreads();
    const int r = x - v + (warp > 0 ? sh[warp - 1] : 0);
    *total = sh[KEY_T / 32 - 1];
    return r;
}

// ---- 2a. per-cell totals (and per-block sums of them) -------------------------
__global__ void __launch_bounds__(KEY_T) k_sort_totals(const SortParams S) {
    __shared__ int sh[KEY_T / 32];
    const int s = blockIdx.y;
    const int key = blockIdx.x * KEY_T + threadIdx.x;
    int tot = 0;
    if (key < S.Nx) {
        int u0, u1;
        covering(S, s, key, u0, u1);
        for (int u = u0; u <= u1; ++u) {
            const int l = key - (S.units.lo[u] - S.k);
            if (l >= 0 && l < ESC) tot += S.cnt[static_cast<size_t>(u) * SSTR + l];
        }
        S.keycount[s][key] = tot;
    }
    const int b = block_sum_int(tot, sh);
    if (threadIdx.x == 0) S.blocksum[s][blockIdx.x] = b;
}

// per-block sums of key counts filled by atomics (fresh load)
__global__ void __launch_bounds__(KEY_T) k_block_sums(const SortParams S) {
    __shared__ int sh[KEY_T / 32];
    const int s = blockIdx.y;
    const int key = blockIdx.x * KEY_T + threadIdx.x;
    const int v = key < S.Nx ? S.keycount[s][key] : 0;
    const int b = block_sum_int(v, sh);
    if (threadIdx.x == 0) S.blocksum[s][blockIdx.x] = b;
}

// exclusive scan of n ints held contiguously, by one block of SCAN_T threads
// (each thread a contiguous range); writes out[0..n) and returns the total
__device__ int block_scan_ranges(const int32_t* in, int32_t* out, int n, int* sh) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (n + SCAN_T - 1) / SCAN_T;
    const int a = min(n, tid * per), b = min(n, a + per);
    int sum = 0;
    for (int i = a; i < b; ++i) sum += in[i];
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = sh[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;
    }
    __syncthreads();
    int run = x - sum + (warp > 0 ? sh[warp - 1] : 0);
    for (int i = a; i < b; ++i) {
        const int v = in[i];
        out[i] = run;
        run += v;
    }
    const int total = sh[SCAN_T / 32 - 1];
    __syncthreads();
    return total;
}

// ---- 2b. scan of the per-block key sums; escape offsets of the units ----------
// One block per species.  blockstart[s][b] = keys before block b; keystart[s][Nx]
// = active particles; esc_off[u] = destination of unit u's first escaped
// particle (after all active ones); meta[2+s] = escapes since the last sort.
__global__ void __launch_bounds__(SCAN_T) k_scan_blocks(const SortParams S, int nkb, int with_units) {
    __shared__ int sh[SCAN_T / 32];
    const int s = blockIdx.x;
    const int act = block_scan_ranges(S.blocksum[s], S.blockstart[s], nkb, sh);
    if (threadIdx.x == 0) S.keystart[s][S.Nx] = act;
    if (!with_units) return;
    const int ub = unit_base(S.units, s), nu = S.units.count[1 + s];
    const int esc = block_scan_ranges(S.esc_cnt + ub, S.esc_off + ub, nu, sh);
    for (int u = threadIdx.x; u < nu; u += SCAN_T) S.esc_off[ub + u] += act;
    if (threadIdx.x == 0) S.meta[2 + s] = esc;
}

// keystart[s][key] from the block starts and a block scan of the key counts
__global__ void __launch_bounds__(KEY_T) k_keystart(const SortParams S) {
    __shared__ int sh[KEY_T / 32];
    const int s = blockIdx.y;
    const int key = blockIdx.x * KEY_T + threadIdx.x;
    const int v = key < S.Nx ? S.keycount[s][key] : 0;
    int total;
    const int r = block_excl_scan(v, sh, &total);
    if (key < S.Nx) S.keystart[s][key] = S.blockstart[s][blockIdx.x] + r;
}

// ---- 2c. cell starts and the destination of every (unit, cell) pair ----------
__global__ void __launch_bounds__(KEY_T) k_sort_offsets(const SortParams S) {
    __shared__ int sh[KEY_T / 32];
    const int s = blockIdx.y;
    const int key = blockIdx.x * KEY_T + threadIdx.x;
    const int v = key < S.Nx ? S.keycount[s][key] : 0;
    int total;
    const int r = block_excl_scan(v, sh, &total);
    if (key >= S.Nx) return;
    int run = S.blockstart[s][blockIdx.x] + r;
    S.keystart[s][key] = run;
    int u0, u1;
    covering(S, s, key, u0, u1);
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

// ---- 4. unit table from sorted cells ------------------------------------------
// 4a. units per tile (TILE cells, at most UNIT_P particles a unit), scanned
// per species by one block: tile_first[s][t] = first unit of tile t.
__global__ void __launch_bounds__(SCAN_T) k_tile_units(const SortParams S) {
    __shared__ int sh[SCAN_T / 32];
    const int ntiles = (S.Nx + TILE - 1) / TILE;
    int base = 0;
    for (int s = 0; s < 2; ++s) {
        const int32_t* ks = S.keystart[s];
        for (int t = threadIdx.x; t < ntiles; t += SCAN_T) {
            const int ts = ks[t * TILE], te = ks[min((t + 1) * TILE, S.Nx)];
            S.tile_n[s][t] = (te - ts + UNIT_P - 1) / UNIT_P;
        }
        __syncthreads();
        const int nu = block_scan_ranges(S.tile_n[s], S.tile_first[s], ntiles, sh);
        if (threadIdx.x == 0) {
            S.tile_first[s][ntiles] = nu;
            S.units.count[1 + s] = nu;
            S.meta[s] = ks[S.Nx];  // active particles at this sort
        }
        base += nu;
        __syncthreads();
    }
    if (threadIdx.x == 0) S.units.count[0] = min(base, S.max_units);
}

// 4b. one thread per unit
__global__ void k_fill_units(const SortParams S) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= S.units.count[0]) return;
    const int n0 = S.units.count[1];
    const int s = u < n0 ? 0 : 1;
    const int v = u - (s ? n0 : 0);
    const int ntiles = (S.Nx + TILE - 1) / TILE;
    const int32_t* tf = S.tile_first[s];
    int l = 0, r = ntiles;  // last tile t with tf[t] <= v
    while (r - l > 1) {
        const int m = (l + r) >> 1;
        if (tf[m] <= v) l = m; else r = m;
    }
    const int t = l;
    const int32_t* ks = S.keystart[s];
    const int ts = ks[t * TILE], te = ks[min((t + 1) * TILE, S.Nx)];
    const int a = ts + (v - tf[t]) * UNIT_P;
    const int b = min(a + UNIT_P, te);
    S.units.species[u] = s;
    S.units.start[u] = a;
    S.units.end[u] = b;
    S.units.lo[u] = S.dst[s].cell[a];
    S.units.hi[u] = S.dst[s].cell[b - 1];
}

// ---- histogram of sorted, freshly loaded particles ---------------------------
// warp-aggregated: lanes holding the same cell add their count once
__global__ void k_hist(const SortParams S) {
    const int s = blockIdx.y;
    const int64_t n = S.n[s];
    const int lane = threadIdx.x & 31;
    for (int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); b < n;
         b += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = b + lane;
        const int c = i < n ? S.dst[s].cell[i] : -1;
        const unsigned peers = __match_any_sync(FULL, c);
        if (c >= 0 && c < S.Nx && lane == __ffs(peers) - 1) atomicAdd(&S.keycount[s][c], __popc(peers));
    }
}

}  // namespace

void launch_sort(const SortParams& S, int n_unit_blocks, cudaStream_t st, int* launches) {
    const int kb = (S.Nx + KEY_T - 1) / KEY_T;
    k_sort_count<<<n_unit_blocks, SORT_T, 0, st>>>(S);
    k_sort_totals<<<dim3(kb, 2), KEY_T, 0, st>>>(S);
    k_scan_blocks<<<2, SCAN_T, 0, st>>>(S, kb, 1);
    k_sort_offsets<<<dim3(kb, 2), KEY_T, 0, st>>>(S);
    k_sort_scatter<<<n_unit_blocks + 64, SORT_T, 0, st>>>(S);
    k_tile_units<<<1, SCAN_T, 0, st>>>(S);
    k_fill_units<<<(S.max_units + 255) / 256, 256, 0, st>>>(S);
    *launches += 7;
}

void launch_build_units_from_sorted(const SortParams& S, cudaStream_t st, int* launches) {
    const int kb = (S.Nx + KEY_T - 1) / KEY_T;
    cudaMemsetAsync(S.keycount[0], 0, sizeof(int32_t) * (S.Nx + 2), st);
    cudaMemsetAsync(S.keycount[1], 0, sizeof(int32_t) * (S.Nx + 2), st);
    k_hist<<<dim3(256, 2), 256, 0, st>>>(S);
    k_block_sums<<<dim3(kb, 2), KEY_T, 0, st>>>(S);
    k_scan_blocks<<<2, SCAN_T, 0, st>>>(S, kb, 0);
    k_keystart<<<dim3(kb, 2), KEY_T, 0, st>>>(S);
    k_tile_units<<<1, SCAN_T, 0, st>>>(S);
    k_fill_units<<<(S.max_units + 255) / 256, 256, 0, st>>>(S);
    *launches += 6;
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
