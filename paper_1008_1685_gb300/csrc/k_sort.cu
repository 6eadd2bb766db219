// Periodic cell sort of the particles of every run of a batch, and the unit
// table built from it.
//
// The sort is a stable counting sort by cell (a particle frozen at a wall
// sorts under its last cell).  It exploits what the push guarantees: a
// particle moves less than one cell per step, so k steps after the last sort
// every particle of unit u has a cell in [lo_u - k, hi_u + k].  Hence, for
// every active run and species of the batch, in one launch per phase:
//   1. each unit counts its particles per cell of that window (warp-aggregated
//      shared-memory integer atomics);
//   2. for each cell the units whose window covers it form a contiguous range
//      (lo and hi are sorted within a run and species), found by binary
//      search; the per-cell totals are scanned into the new cell starts, and
//      every (unit, cell) pair gets its destination offset in unit order;
//   3. each unit scatters its particles, ranking equal cells in index order
//      (each warp owns a contiguous slice; warp match ranks within a warp and
//      per-warp counts combined in warp order), so the result does not depend
//      on scheduling;
//   4. the unit table is rebuilt from the sorted cells: tiles of TILE cells,
//      split into chunks of at most unit_p particles, except that an aligned
//      group of GROUP consecutive tiles holding at most unit_p particles
//      together forms one unit, or else an aligned half group that does
//      (sparse regions would otherwise give many nearly empty units).
// Every particle is read once and written once; the cell array is read once
// more for the counts.
#include <algorithm>
#include <climits>

#include "picrr_internal.cuh"

namespace picrr {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int SORT_T = 256;
constexpr int SCAN_T = 1024;

// sort key of a stored cell: frozen particles (cell = -1 - k) sort under k
__device__ __forceinline__ int key_of(int c) { return c < 0 ? -1 - c : c; }

// ---- 1. per-unit window counts -------------------------------------------------
__global__ void __launch_bounds__(SORT_T) k_sort_count(const SortParams S) {
    __shared__ int cnt[SSTR];
    const int u = blockIdx.x;
    if (u >= S.units.count[0]) return;
    const RunDev& R = S.runs[S.units.run[u]];
    if (!R.active) return;  // a run that ended keeps its particles where they are
    const int s = S.units.species[u];
    const int start = S.units.start[u], end = S.units.end[u];
    const int wb = S.units.lo[u] - S.k;
    const int L = S.units.hi[u] + S.k + 1 - wb;
    for (int i = threadIdx.x; i < SSTR; i += SORT_T) cnt[i] = 0;
    __syncthreads();
    const int32_t* cell = R.sp[s][S.cur].cell;
    const int lane = threadIdx.x & 31;
    constexpr int U = 4;  // loads in flight per thread
    for (int i0 = start; i0 < end; i0 += U * SORT_T) {  // block-uniform trip count
        int c[U];
#pragma unroll
        for (int m = 0; m < U; ++m) {
            const int i = i0 + m * SORT_T + threadIdx.x;
            c[m] = i < end ? cell[i] : INT32_MIN;
        }
#pragma unroll
        for (int m = 0; m < U; ++m) {
            int l = -1;
            if (c[m] != INT32_MIN) {
                l = key_of(c[m]) - wb;
                if (!(l >= 0 && l < L && l < SSTR)) {
                    atomicOr(S.status, ST_WINDOW);
                    l = -1;
                }
            }
            // lanes with the same cell add their count once
            const unsigned peers = __match_any_sync(FULL, l);
            if (l >= 0 && lane == __ffs(peers) - 1) atomicAdd(&cnt[l], __popc(peers));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < L; i += SORT_T) S.cnt[static_cast<size_t>(u) * SSTR + i] = cnt[i];
}

// Units of run `run`, species s whose window covers cell `key`: [u0, u1].
__device__ void covering(const SortParams& S, int run, int s, int key, int& u0, int& u1) {
    const int p = 2 * run + s;
    const int b = S.rs_units[2 * S.nruns + p], n = S.rs_units[p];
    int l = 0, r = n;  // first u with hi + k >= key
    while (l < r) {
        const int m = (l + r) >> 1;
        if (S.units.hi[b + m] + S.k >= key) r = m; else l = m + 1;
    }
    u0 = b + l;
    l = 0;
    r = n;  // last u with lo - k <= key
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

// exclusive scan of v over the block (KEY_T threads)
__device__ __forceinline__ int block_excl_scan(int v, int* sh) {
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
    return x - v + (warp > 0 ? sh[warp - 1] : 0);
}

// exclusive scan of n ints by one block of SCAN_T threads (each thread a
// contiguous range); writes out[0..n) and returns the total
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

// ---- 2a. per-cell totals (and per-block sums of them) --------------------------
// grid (key blocks of the largest run, runs, species)
__global__ void __launch_bounds__(KEY_T) k_sort_totals(const SortParams S) {
    __shared__ int sh[KEY_T / 32];
    const RunDev& R = S.runs[blockIdx.y];
    const int s = blockIdx.z;
    if (!R.active || blockIdx.x * KEY_T >= R.Nx) return;  // block-uniform
    const int key = blockIdx.x * KEY_T + threadIdx.x;
    int tot = 0;
    if (key < R.Nx) {
        int u0, u1;
        covering(S, blockIdx.y, s, key, u0, u1);
        for (int u = u0; u <= u1; ++u) {
            const int l = key - (S.units.lo[u] - S.k);
            if (l >= 0 && l < SSTR) tot += S.cnt[static_cast<size_t>(u) * SSTR + l];
        }
        R.keycount[s][key] = tot;
    }
    const int b = block_sum_int(tot, sh);
    if (threadIdx.x == 0) R.blocksum[s][blockIdx.x] = b;
}

// ---- 2b. scan of the per-block sums, one block per (run, species) --------------
__global__ void __launch_bounds__(SCAN_T) k_scan_blocks(const SortParams S) {
    __shared__ int sh[SCAN_T / 32];
    const RunDev& R = S.runs[blockIdx.x];
    const int s = blockIdx.y;
    if (!R.active) return;
    const int nkb = (R.Nx + KEY_T - 1) / KEY_T;
    const int total = block_scan_ranges(R.blocksum[s], R.blockstart[s], nkb, sh);
    if (threadIdx.x == 0) R.keystart[s][R.Nx] = total;
}

// ---- 2c. cell starts and the destination of every (unit, cell) pair -------------
__global__ void __launch_bounds__(KEY_T) k_sort_offsets(const SortParams S) {
    __shared__ int sh[KEY_T / 32];
    const RunDev& R = S.runs[blockIdx.y];
    const int s = blockIdx.z;
    if (!R.active || blockIdx.x * KEY_T >= R.Nx) return;
    const int key = blockIdx.x * KEY_T + threadIdx.x;
    const int v = key < R.Nx ? R.keycount[s][key] : 0;
    const int r = block_excl_scan(v, sh);
    if (key >= R.Nx) return;
    int run = R.blockstart[s][blockIdx.x] + r;
    R.keystart[s][key] = run;
    int u0, u1;
    covering(S, blockIdx.y, s, key, u0, u1);
    for (int u = u0; u <= u1; ++u) {
        const int l = key - (S.units.lo[u] - S.k);
        if (l >= 0 && l < SSTR) {
            const size_t q = static_cast<size_t>(u) * SSTR + l;
            S.offs[q] = run;
            run += S.cnt[q];
        }
    }
}


// ---- 3. stable scatter ----------------------------------------------------------
// Each warp owns one contiguous slice of the unit's particles.  Pass 1 counts
// the slice's particles per cell (warp match; only the warp writes its row);
// the rows are then turned into per-warp destination starts (unit offset plus
// the counts of the warps before, in warp order); pass 2 walks the slice
// again in order and places each particle at its warp's running start plus
// its rank among the lanes with the same cell.  Equal cells therefore keep
// index order, with two block barriers per unit.
constexpr int SC_W = SORT_T / 32;
constexpr int SC_U = 4;  // slice rows of 32 particles in flight per pass step

__device__ __forceinline__ int window_key(const int32_t* cell, int i, int we, int wb) {
    if (i >= we) return -1;
    const int l = key_of(cell[i]) - wb;
    return (l >= 0 && l < SSTR) ? l : -1;  // out of window cannot happen (counted as an error)
}

__global__ void __launch_bounds__(SORT_T) k_sort_scatter(const SortParams S) {
    __shared__ int row[SC_W][SSTR];
    const int u = blockIdx.x;
    if (u >= S.units.count[0]) return;
    const RunDev& R = S.runs[S.units.run[u]];
    if (!R.active) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s = S.units.species[u];
    const int start = S.units.start[u], end = S.units.end[u];
    const int wb = S.units.lo[u] - S.k;
    const DevSpecies src = R.sp[s][S.cur];
    const DevSpecies dst = R.sp[s][1 - S.cur];
    const int per = (end - start + SC_W - 1) / SC_W;
    const int ws = min(end, start + warp * per), we = min(end, ws + per);
    for (int i = tid; i < SC_W * SSTR; i += SORT_T) (&row[0][0])[i] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    // pass 1: this warp's counts per cell
    for (int i0 = ws; i0 < we; i0 += 32 * SC_U) {  // warp-uniform
        int key[SC_U];
#pragma unroll
        for (int m = 0; m < SC_U; ++m) key[m] = window_key(src.cell, i0 + 32 * m + lane, we, wb);
#pragma unroll
        for (int m = 0; m < SC_U; ++m) {
            const unsigned peers = __match_any_sync(FULL, key[m]);
            if (key[m] >= 0 && lane == __ffs(peers) - 1) row[warp][key[m]] += __popc(peers);
            __syncwarp();
        }
    }
    __syncthreads();
    // per cell of the window: destination start of each warp's particles, in warp order
    const int L = S.units.hi[u] + S.k + 1 - wb;
    for (int l = tid; l < L && l < SSTR; l += SORT_T) {
        int run = S.offs[static_cast<size_t>(u) * SSTR + l];
#pragma unroll
        for (int w = 0; w < SC_W; ++w) {
            const int c = row[w][l];
            row[w][l] = run;
            run += c;
        }
    }
    __syncthreads();
    // pass 2: place the slice's particles in order
    for (int i0 = ws; i0 < we; i0 += 32 * SC_U) {  // warp-uniform
        int cl[SC_U], id[SC_U];
        float of[SC_U], x[SC_U], y[SC_U], z[SC_U];
#pragma unroll
        for (int m = 0; m < SC_U; ++m) {
            const int i = i0 + 32 * m + lane;
            if (i < we) {
                cl[m] = src.cell[i];
                of[m] = src.off[i];
                x[m] = src.px[i];
                y[m] = src.py[i];
                z[m] = src.pz[i];
                id[m] = src.id[i];
            }
        }
#pragma unroll
        for (int m = 0; m < SC_U; ++m) {
            const int i = i0 + 32 * m + lane;
            int key = -1;
            if (i < we) {
                const int l = key_of(cl[m]) - wb;
                key = (l >= 0 && l < SSTR) ? l : -1;
            }
            const unsigned peers = __match_any_sync(FULL, key);
            const int d = key >= 0 ? row[warp][key] + __popc(peers & lt) : -1;
            __syncwarp();
            if (key >= 0 && lane == __ffs(peers) - 1) row[warp][key] += __popc(peers);
            __syncwarp();
            if (d >= 0) {
                dst.cell[d] = cl[m];
                dst.off[d] = of[m];
                dst.px[d] = x[m];
                dst.py[d] = y[m];
                dst.pz[d] = z[m];
                dst.id[d] = id[m];
            }
        }
    }
}

// ---- 4. unit table from sorted cells -------------------------------------------
// 4a. units per tile of one (run, species), scanned: tile_first[t] = first
// unit of tile t within the pair; rs_units[2 r + s] = the pair's units.
__global__ void __launch_bounds__(SCAN_T) k_tile_units(const SortParams S) {
    __shared__ int sh[SCAN_T / 32];
    const int r = blockIdx.x, s = blockIdx.y;
    const RunDev& R = S.runs[r];
    if (!R.active || R.n[s] == 0) {
        if (threadIdx.x == 0) S.rs_units[2 * r + s] = 0;
        return;
    }
    const int ntiles = (R.Nx + TILE - 1) / TILE;
    const int32_t* ks = R.keystart[s];
    for (int t = threadIdx.x; t < ntiles; t += SCAN_T) {
        // an aligned group of GROUP tiles holding at most unit_p particles is one
        // unit, counted on its first tile; otherwise each aligned half group of
        // GROUP / 2 tiles that holds at most unit_p is one unit; otherwise each
        // tile is split on its own
        const int g0 = (t / GROUP) * SPAN;
        const int gn = ks[min(g0 + SPAN, R.Nx)] - ks[g0];
        const int h0 = (t / (GROUP / 2)) * (SPAN / 2);
        const int hn = ks[min(h0 + SPAN / 2, R.Nx)] - ks[h0];
        int n;
        if (gn <= S.unit_p) {
            n = (t % GROUP == 0 && gn > 0) ? 1 : 0;
        } else if (hn <= S.unit_p) {
            n = (t % (GROUP / 2) == 0 && hn > 0) ? 1 : 0;
        } else {
            const int ts = ks[t * TILE], te = ks[min((t + 1) * TILE, R.Nx)];
            n = (te - ts + S.unit_p - 1) / S.unit_p;
        }
        R.tile_n[s][t] = n;
    }
    __syncthreads();
    const int nu = block_scan_ranges(R.tile_n[s], R.tile_first[s], ntiles, sh);
    if (threadIdx.x == 0) {
        R.tile_first[s][ntiles] = nu;
        S.rs_units[2 * r + s] = nu;
    }
}

// 4b. unit bases of every (run, species) pair, in run-major order
__global__ void __launch_bounds__(SCAN_T) k_unit_bases(const SortParams S) {
    __shared__ int sh[SCAN_T / 32];
    const int np = 2 * S.nruns;
    const int total = block_scan_ranges(S.rs_units, S.rs_units + np, np, sh);
    if (threadIdx.x == 0) S.units.count[0] = min(total, S.max_units);
}

// 4c. one thread per unit; the sorted particles are in buffer `ubuf`
__global__ void k_fill_units(const SortParams S, int ubuf) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= S.units.count[0]) return;
    const int np = 2 * S.nruns;
    const int32_t* first = S.rs_units + np;  // exclusive scan of the pair counts
    int l = 0, r = np;  // last pair with first[p] <= u and a unit count > 0
    while (r - l > 1) {
        const int m = (l + r) >> 1;
        if (first[m] <= u) l = m; else r = m;
    }
    while (S.rs_units[l] == 0 && l > 0) --l;  // skip empty pairs sharing the same start
    const int run = l >> 1, s = l & 1;
    const RunDev& R = S.runs[run];
    const int v = u - first[l];
    const int ntiles = (R.Nx + TILE - 1) / TILE;
    const int32_t* tf = R.tile_first[s];
    int a0 = 0, b0 = ntiles;  // last tile t with tf[t] <= v
    while (b0 - a0 > 1) {
        const int m = (a0 + b0) >> 1;
        if (tf[m] <= v) a0 = m; else b0 = m;
    }
    const int t = a0;
    const int32_t* ks = R.keystart[s];
    const int g0 = (t / GROUP) * SPAN;
    const int gs = ks[g0], ge = ks[min(g0 + SPAN, R.Nx)];
    const int h0 = (t / (GROUP / 2)) * (SPAN / 2);
    const int hs = ks[h0], he = ks[min(h0 + SPAN / 2, R.Nx)];
    int a, b;
    if (ge - gs <= S.unit_p) {  // the whole group (t is its first tile)
        a = gs;
        b = ge;
    } else if (he - hs <= S.unit_p) {  // the half group (t is its first tile)
        a = hs;
        b = he;
    } else {
        const int ts = ks[t * TILE], te = ks[min((t + 1) * TILE, R.Nx)];
        a = ts + (v - tf[t]) * S.unit_p;
        b = min(a + S.unit_p, te);
    }
    const int32_t* cell = R.sp[s][ubuf].cell;
    S.units.run[u] = run;
    S.units.species[u] = s;
    S.units.start[u] = a;
    S.units.end[u] = b;
    S.units.lo[u] = key_of(cell[a]);
    S.units.hi[u] = key_of(cell[b - 1]);
}

// ---- histogram of already sorted particles (fresh load) -------------------------
// grid (blocks, runs, species); warp-aggregated
__global__ void k_hist(const SortParams S) {
    const RunDev& R = S.runs[blockIdx.y];
    const int s = blockIdx.z;
    if (!R.active) return;
    const int n = R.n[s];
    const int lane = threadIdx.x & 31;
    const int32_t* cell = R.sp[s][S.cur].cell;
    for (int b = blockIdx.x * blockDim.x + (threadIdx.x & ~31); b < n; b += gridDim.x * blockDim.x) {
        const int i = b + lane;
        const int c = i < n ? key_of(cell[i]) : -1;
        const unsigned peers = __match_any_sync(FULL, c);
        if (c >= 0 && c < R.Nx && lane == __ffs(peers) - 1) atomicAdd(&R.keycount[s][c], __popc(peers));
    }
}

__global__ void __launch_bounds__(KEY_T) k_block_sums(const SortParams S) {
    __shared__ int sh[KEY_T / 32];
    const RunDev& R = S.runs[blockIdx.y];
    const int s = blockIdx.z;
    if (!R.active || blockIdx.x * KEY_T >= R.Nx) return;
    const int key = blockIdx.x * KEY_T + threadIdx.x;
    const int v = key < R.Nx ? R.keycount[s][key] : 0;
    const int b = block_sum_int(v, sh);
    if (threadIdx.x == 0) R.blocksum[s][blockIdx.x] = b;
}

__global__ void __launch_bounds__(KEY_T) k_keystart(const SortParams S) {
    __shared__ int sh[KEY_T / 32];
    const RunDev& R = S.runs[blockIdx.y];
    const int s = blockIdx.z;
    if (!R.active || blockIdx.x * KEY_T >= R.Nx) return;
    const int key = blockIdx.x * KEY_T + threadIdx.x;
    const int v = key < R.Nx ? R.keycount[s][key] : 0;
    const int r = block_excl_scan(v, sh);
    if (key < R.Nx) R.keystart[s][key] = R.blockstart[s][blockIdx.x] + r;
}

__global__ void k_zero_keycount(const SortParams S) {
    const RunDev& R = S.runs[blockIdx.y];
    const int s = blockIdx.z;
    if (!R.active) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < R.Nx + 2; i += gridDim.x * blockDim.x)
        R.keycount[s][i] = 0;
}

// ---- radiated energy per run: sum of its electron units, fixed order ------------
__global__ void __launch_bounds__(1024) k_rad_flush(const RunDev* runs, const int32_t* rs_units, double* part) {
    __shared__ double sred[32];
    const RunDev& R = runs[blockIdx.x];
    if (!R.active) return;
    const int b = rs_units[2 * gridDim.x + 2 * blockIdx.x], n = rs_units[2 * blockIdx.x];  // electron units
    const int t = threadIdx.x;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int i = t;
    for (; i + 3 * 1024 < n; i += 4 * 1024) {
        a0 += part[b + i];
        a1 += part[b + i + 1024];
        a2 += part[b + i + 2048];
        a3 += part[b + i + 3072];
        part[b + i] = part[b + i + 1024] = part[b + i + 2048] = part[b + i + 3072] = 0.0;
    }
    for (; i < n; i += 1024) {
        a0 += part[b + i];
        part[b + i] = 0.0;
    }
    double v = (a0 + a1) + (a2 + a3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if ((t & 31) == 0) sred[t >> 5] = v;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < 32; ++w) s += sred[w];
        R.tally[0] += s;
    }
}

}  // namespace

void launch_sort(const SortParams& S, cudaStream_t st, int* launches) {
    const dim3 kg(S.kb_max, S.nruns, 2);
    k_sort_count<<<S.max_units, SORT_T, 0, st>>>(S);
    k_sort_totals<<<kg, KEY_T, 0, st>>>(S);
    k_scan_blocks<<<dim3(S.nruns, 2), SCAN_T, 0, st>>>(S);
    k_sort_offsets<<<kg, KEY_T, 0, st>>>(S);
    k_sort_scatter<<<S.max_units, SORT_T, 0, st>>>(S);
    k_tile_units<<<dim3(S.nruns, 2), SCAN_T, 0, st>>>(S);
    k_unit_bases<<<1, SCAN_T, 0, st>>>(S);
    k_fill_units<<<(S.max_units + 255) / 256, 256, 0, st>>>(S, 1 - S.cur);
    *launches += 8;
}

void launch_build_units(const SortParams& S, cudaStream_t st, int* launches) {
    const dim3 kg(S.kb_max, S.nruns, 2);
    k_zero_keycount<<<dim3(64, S.nruns, 2), 256, 0, st>>>(S);
    k_hist<<<dim3(256, S.nruns, 2), 256, 0, st>>>(S);
    k_block_sums<<<kg, KEY_T, 0, st>>>(S);
    k_scan_blocks<<<dim3(S.nruns, 2), SCAN_T, 0, st>>>(S);
    k_keystart<<<kg, KEY_T, 0, st>>>(S);
    k_tile_units<<<dim3(S.nruns, 2), SCAN_T, 0, st>>>(S);
    k_unit_bases<<<1, SCAN_T, 0, st>>>(S);
    k_fill_units<<<(S.max_units + 255) / 256, 256, 0, st>>>(S, S.cur);
    *launches += 8;
}

void launch_rad_flush(const RunDev* runs, int nruns, const int32_t* rs_units, double* rad_part, cudaStream_t st) {
    k_rad_flush<<<nruns, 1024, 0, st>>>(runs, rs_units, rad_part);
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
