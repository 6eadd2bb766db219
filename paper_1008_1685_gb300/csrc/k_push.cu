// Fused field gather + Boris push + Landau-Lifshitz radiation-reaction kick
// + move + charge-conserving deposit (the particle part of one PIC step).
//
// One CTA per work unit (at most unit_p consecutive particles of one species
// whose cells at the last sort lie in one tile, or in one aligned group or
// half group of sparse tiles holding at most unit_p particles; unit_p is a
// shape of the batch).
// Because cfl < 1 a particle moves less than one cell per step, so k steps
// after the sort every particle of the unit lies in [lo - k, hi + k]; the CTA
// stages the fields of the window [lo - k - 1, hi + k + 2] into shared memory
// (with 4 particles per thread: plain loads into a gather-ready layout; with 2:
// one bulk TMA copy per component, completing on one mbarrier), streams the
// particles (structure of arrays) with 128- or 64-bit evict-first loads and
// stores, and accumulates the unit's current in shared memory.
//
// Deposit: a particle that moves from bin b (cell at x^n) to bin b + d,
// d in {-1, 0, 1}, touches Jy and Jz on at most three nodes and Jx on at most
// two half nodes, all within the stencil anchored at a = min(b, b + d): one
// record of eight values per particle (the 1D Esirkepov split for linear
// shapes: the old bin's share up to the crossing point, the new bin's after
// it).  Determinism: a thread first adds the records of its successive
// particles that share an anchor, in a fixed order; the record is then
// converted to 32-bit fixed point and added to the unit's window in shared
// memory with integer atomics, which hold exact 64-bit sums as pairs of 32-bit
// words (when all lanes of a warp hold the same anchor, as in dense plasma,
// the lanes are first summed exactly by an integer warp reduction).  At the
// end the window is shifted to the 64-bit scale of the accumulators and added
// to global memory with integer atomics.  Integer addition is exact and
// associative, so the result does not depend on the order in which lanes,
// warps or CTAs arrive.
#include "picrr_internal.cuh"

namespace picrr {

namespace {

constexpr unsigned FULL = 0xffffffffu;

#ifndef PICRR_THIN_PER_CELL
#define PICRR_THIN_PER_CELL 8
#endif
// Units with fewer particles per cell than this (thinly spread plasma, where
// nearly every lane of a warp holds its own anchor) skip the warp-wide test
// of warp_add altogether: every lane adds its records by itself.
constexpr int kThinPerCell = PICRR_THIN_PER_CELL;

// The unit's current window in shared memory holds exact 64-bit integer sums
// (in the 2^lscale units of the records) as two 32-bit words, lo (unsigned)
// and hi (signed): value = hi * 2^32 + lo.  A signed 32-bit term t is added
// with a 32-bit atomic on lo, which returns the old word: the addition
// wrapped (carried) iff the new word is below the old one, and hi then gets
// sign(t) + carry (-1, 0 or +1; nothing in most cases).  Every carry is seen by
// exactly one adder, so the pair always holds the exact sum, in any order.
// (A 64-bit shared-memory atomic runs at a sixth of the 32-bit rate.)
struct Window {
    unsigned lo[3][WMAX];  // Jx (half nodes), Jy, Jz (nodes)
    int hi[3][WMAX];
};

__device__ __forceinline__ void win_add(Window& w, int comp, int at, int t) {
    const unsigned old = atomicAdd(&w.lo[comp][at], static_cast<unsigned>(t));
    const int h = (t < 0 ? -1 : 0) + (old + static_cast<unsigned>(t) < old ? 1 : 0);
    if (h) atomicAdd(&w.hi[comp][at], h);
}

// Position of value q of a stencil record anchored at key: q 0..2 are Jy at
// key+q, 3..5 Jz at key+q-3, 6 and 7 Jx at half nodes key, key+1.
__device__ __forceinline__ int rec_comp(int q) { return q < 3 ? 1 : (q < 6 ? 2 : 0); }
__device__ __forceinline__ int rec_at(int key, int q) { return key + (q < 3 ? q : (q < 6 ? q - 3 : q - 6)); }

// One lane's record added by itself: each nonzero value rounded to 32-bit
// fixed point (records are kept in the window's units, |value| < 2^26).
__device__ __forceinline__ void lane_add(int key, const float (&v)[8], Window& w) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int t = __float2int_rn(v[q]);
        if (t) win_add(w, rec_comp(q), rec_at(key, q), t);
    }
}

// One stencil record per lane (key < 0: none).  When every lane holds the
// same anchor (dense plasma), the records are summed exactly in 32-bit fixed
// point (|value| < 2^26 per lane, so the warp sum fits) by one integer warp
// reduction per value and lanes 0..7 add the eight sums (the large run's push
// 0.463 -> 0.450 ms against eight adds by lane 0); otherwise every lane adds
// its own record.  (A reduction over lanes grouped by anchor runs once per
// distinct anchor, which costs more than the lanes' own atomics as soon as
// the warp holds two.)
__device__ __forceinline__ void warp_add(int key, const float (&v)[8], Window& w) {
    const int k0 = __shfl_sync(FULL, key, 0);
    if (__all_sync(FULL, key == k0)) {
        if (k0 >= 0) {
            // lane q (q < 8) adds the warp sum of value q: eight distinct words
            const int lane = threadIdx.x & 31;
            int mine = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int t = __reduce_add_sync(FULL, __float2int_rn(v[q]));
                mine = lane == q ? t : mine;
            }
            if (lane < 8 && mine) win_add(w, rec_comp(lane), rec_at(k0, lane), mine);
        }
    } else {
        // lanes 2m and 2m+1 that hold the same anchor: the even lane adds the
        // pair's integer sum (exact: |sum| < 2^27), the odd lane nothing, which
        // halves the same-word atomics of lanes that share an anchor (the
        // 256-run scan's late-phase push 0.542 -> 0.530 ms); the window's sums
        // are the same integers
        const int lane = threadIdx.x & 31;
        const int kn = __shfl_xor_sync(FULL, key, 1);
        const bool pair = key >= 0 && kn == key;
        int t[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int tq = __float2int_rn(v[q]);
            const int tn = __shfl_xor_sync(FULL, tq, 1);
            t[q] = pair ? tq + tn : tq;
        }
        if (key >= 0 && !(pair && (lane & 1))) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (t[q]) win_add(w, rec_comp(q), rec_at(key, q), t[q]);
        }
    }
}

// Reciprocal square root and quotient for arguments x >= 1 (1 + p^2, 1 + t^2,
// sums of Lorentz factors): the approximate hardware forms with flush of
// subnormal inputs, which never applies to such x, so the subnormal checks of
// the general forms are dropped (2.6 % of the push time on dense foils).
__device__ __forceinline__ float rsqrt_ge1(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float div_ge1(float a, float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return a * y;
}

__device__ __forceinline__ int comp(const int4& a, int j) { return j == 0 ? a.x : j == 1 ? a.y : j == 2 ? a.z : a.w; }
__device__ __forceinline__ float comp(const float4& a, int j) {
    return j == 0 ? a.x : j == 1 ? a.y : j == 2 ? a.z : a.w;
}
__device__ __forceinline__ int comp(const int2& a, int j) { return j == 0 ? a.x : a.y; }
__device__ __forceinline__ float comp(const float2& a, int j) { return j == 0 ? a.x : a.y; }

// A thread takes W consecutive particles per round (one W x 4-byte slot of each
// array).  W = 4: 128-bit loads and stores, fewest instructions per particle,
// for dense foils.  W = 2: 64-bit, fewer registers and so more warps per SM,
// which hides the latency of deposits that scatter over many cells (thinly
// spread particles).
template <int W>
struct Slot;
template <>
struct Slot<4> {
    using I = int4;
    using F = float4;
    static constexpr int MIN_BLOCKS = 4;
    static __device__ __forceinline__ I empty_i() { return make_int4(-1, -1, -1, -1); }
    static __device__ __forceinline__ F zero_f() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    static __device__ __forceinline__ I pack(const int (&v)[4]) { return make_int4(v[0], v[1], v[2], v[3]); }
    static __device__ __forceinline__ F pack(const float (&v)[4]) { return make_float4(v[0], v[1], v[2], v[3]); }
};
template <>
struct Slot<2> {
    using I = int2;
    using F = float2;
    static constexpr int MIN_BLOCKS = 6;
    static __device__ __forceinline__ I empty_i() { return make_int2(-1, -1); }
    static __device__ __forceinline__ F zero_f() { return make_float2(0.f, 0.f); }
    static __device__ __forceinline__ I pack(const int (&v)[2]) { return make_int2(v[0], v[1]); }
    static __device__ __forceinline__ F pack(const float (&v)[2]) { return make_float2(v[0], v[1]); }
};

// Shared memory of a CTA: the unit's current window and its field window.  With
// 4 particles per thread (dense foils, many particles per window cell) the
// fields are read with plain loads into a layout made for the gather: per node
// i (Ey, Ey[i+1] - Ey, Ez, Ez[i+1] - Ez) and per half node (Ex, dEx, By, dBy)
// and (Bz, dBz), so that a particle's gather is three loads and five FMAs
// (the large run's push 0.451 -> 0.441 ms).  With 2 per thread (thin plasma,
// few particles per cell) the components are copied as they are by bulk TMA,
// and the smaller footprint keeps six CTAs per SM.
template <int W>
struct PushSmem;
template <>
struct PushSmem<4> {
    float4 nd[WMAX];
    float4 hf[WMAX];
    float2 hz[WMAX];
    Window J;
};
template <>
struct PushSmem<2> {
    float F[5][WMAX];
    Window J;
};

template <int W>
__global__ void __launch_bounds__(PUSH_T, Slot<W>::MIN_BLOCKS) k_push_deposit(const PushParams P) {
    using I = typename Slot<W>::I;
    using F = typename Slot<W>::F;
    __shared__ __align__(128) PushSmem<W> sm;
    Window& sJ = sm.J;  // the unit's current: Jx (half nodes), Jy, Jz (nodes) of the window
    __shared__ __align__(8) uint64_t bar;
    __shared__ double sred[PUSH_T / 32];

    const int u = blockIdx.x;
    if (u >= P.units.count[0]) return;  // block-uniform
    const RunDev& R = P.runs[P.units.run[u]];
    if (!R.active) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s = P.units.species[u];
    const int par = static_cast<int>((P.gstep + R.fpar) & 1);
    const int start = P.units.start[u], end = P.units.end[u];
    const int lo = P.units.lo[u], hi = P.units.hi[u];
    const int k = P.k;
    // cells [lo - k, hi + k] plus one neighbour left and two right; particles
    // never leave [0, Nx - 1] (frozen ones are skipped), so the window is also
    // clipped to the grid's cells -1 .. Nx + 1, which the guard elements hold
    const int w0 = max(lo - k - 1, -1), w1 = min(hi + k + 3, R.Nx + 2);
    const int p0 = (w0 + PADF) & ~3;
    const int p1 = (w1 + PADF + 3) & ~3;
    const int L = p1 - p0;
    if (L > WMAX || p0 < 0 || p1 > R.glen) {  // cannot happen for a valid unit table; never copy out of the arrays
        if (tid == 0) atomicOr(P.status, ST_WINDOW);
        return;
    }

    for (int i = tid; i < 3 * WMAX; i += PUSH_T) {
        (&sJ.lo[0][0])[i] = 0u;
        (&sJ.hi[0][0])[i] = 0;
    }
    if (W == 2 && tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    const DevSpecies sp = R.sp[s][P.cur];
    // the unit's particles are read in slots of W, from the aligned slot before
    // `start` to the aligned slot after `end`; the at most W - 1 particles of
    // each neighbouring unit in those slots are never written here
    const int base = start & ~(W - 1);
    const int npw = ((end + W - 1) & ~(W - 1)) - base;
    if constexpr (W == 2) {
        if (tid == 0) {
            mbar_arrive_expect_tx(&bar, 5u * static_cast<uint32_t>(L) * 4u);
#pragma unroll
            for (int c = 0; c < 5; ++c)
                tma_load_1d(&sm.F[c][0], R.F[par][c] + p0, static_cast<uint32_t>(L) * 4u, &bar);
        }
    } else {
        const float* const* Fg = R.F[par];
        for (int i = tid; i < L; i += PUSH_T) {
            const int a = p0 + i, b = p0 + (i + 1 < L ? i + 1 : i);  // both within [p0, p1)
            const float ey = __ldg(Fg[1] + a), ez = __ldg(Fg[2] + a), ex = __ldg(Fg[0] + a);
            const float by = __ldg(Fg[3] + a), bz = __ldg(Fg[4] + a);
            sm.nd[i] = make_float4(ey, __ldg(Fg[1] + b) - ey, ez, __ldg(Fg[2] + b) - ez);
            sm.hf[i] = make_float4(ex, __ldg(Fg[0] + b) - ex, by, __ldg(Fg[3] + b) - by);
            sm.hz[i] = make_float2(bz, __ldg(Fg[4] + b) - bz);
        }
    }

    const float qm = R.qm[s], qw = R.qw[s];
    const float cfl = P.cfl, dt = P.dt, eps = P.eps;
    const float lscale = R.lscale[s];
    const int shift = R.lshift[s];
    const bool rr = s == 0 && R.rr != 0;
    const int Nx = R.Nx;
    const float hq = 0.5f * qm * dt;
    // the record's factors carry the window's power-of-two scale, so that records
    // are summed in its units (an exact scaling: the same bits as scaling each sum)
    const float jxf = qw / cfl * lscale;  // q w dx / dt
    const float hqw = 0.5f * qw * lscale;
    const int nslots = npw / W;
    const int rounds = (nslots + PUSH_T - 1) / PUSH_T;

    if constexpr (W == 2) {
        const bool got = mbar_wait_bounded(&bar, 0);
        if (!__syncthreads_and(got)) {
            if (tid == 0) {
                atomicOr(P.status, ST_TIMEOUT);
                mbar_wait_bounded(&bar, 0);  // let the copy land before the CTA exits
            }
            return;
        }
    } else {
        __syncthreads();
    }

    const bool thin = end - start < kThinPerCell * (hi - lo + 1);  // block-uniform
    float rad = 0.f;
    int rk = -1;  // running stencil record of this thread (anchor rk)
    float rv[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};

    for (int r = 0; r < rounds; ++r) {
        const int slot = r * PUSH_T + tid;
        const int b4 = base + W * slot;
        const bool slot_ok = slot < nslots;
        I c4 = Slot<W>::empty_i();
        F o4 = Slot<W>::zero_f(), x4 = o4, y4 = o4, z4 = o4;
        if (slot_ok) {
            c4 = __ldcs(reinterpret_cast<const I*>(sp.cell + b4));
            o4 = __ldcs(reinterpret_cast<const F*>(sp.off + b4));
            x4 = __ldcs(reinterpret_cast<const F*>(sp.px + b4));
            y4 = __ldcs(reinterpret_cast<const F*>(sp.py + b4));
            z4 = __ldcs(reinterpret_cast<const F*>(sp.pz + b4));
        }
        // the next round's slots into L2 while this round computes, so that its loads
        // wait on L2 rather than HBM: one bulk (TMA) prefetch per array for the whole
        // CTA, with an evict-first policy (the large run's push 0.483 -> 0.463 ms)
        if (tid == 0 && (r + 1) * PUSH_T < nslots) {
            const int n0 = base + W * (r + 1) * PUSH_T;                      // first particle of the next round
            const int n1 = base + W * min((r + 2) * PUSH_T, nslots);         // one past its last
            const int a0 = n0 & ~3, a1 = (n1 + 3) & ~3;                      // 16-byte aligned, within the padded arrays
            const uint32_t bytes = static_cast<uint32_t>(a1 - a0) * 4u;
            uint64_t pol;
            asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
            const void* arrs[5] = {sp.cell + a0, sp.off + a0, sp.px + a0, sp.py + a0, sp.pz + a0};
#pragma unroll
            for (int q = 0; q < 5; ++q)
                asm volatile("cp.async.bulk.prefetch.L2.global.L2::cache_hint [%0], %1, %2;" ::"l"(arrs[q]), "r"(bytes),
                             "l"(pol)
                             : "memory");
        }
        int cn[W];
        float fo[W], qx[W], qy[W], qz[W];
        bool act[W];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const int idx = b4 + j;
            int c = comp(c4, j);
            float f = comp(o4, j);
            float px = comp(x4, j), py = comp(y4, j), pz = comp(z4, j);
            const int lb = c + PADF - p0;  // local bin of the particle's cell
            bool a = slot_ok && idx >= start && idx < end && c >= 0;
            if (a && (lb < 1 || lb > L - 3)) {  // outside the window: leave it, report
                atomicOr(P.status, ST_WINDOW);
                a = false;
            }
            int ka = -1;  // anchor of this particle's stencil record
            float ay = 0.f, az = 0.f, w0 = 0.f, w1 = 0.f, w2 = 0.f, dj0 = 0.f, dj1 = 0.f;
            if (a) {
                // --- linear gather: nodes (Ey, Ez) and half nodes (Ex, By, Bz)
                const float h = f - 0.5f;
                const int jb = h < 0.f ? lb - 1 : lb;
                const float g = h < 0.f ? h + 1.f : h;
                float e_x, e_y, e_z, b_y, b_z;
                if constexpr (W == 4) {
                    const float4 nd = sm.nd[lb];
                    const float4 hf = sm.hf[jb];
                    const float2 hz = sm.hz[jb];
                    e_y = fmaf(f, nd.y, nd.x);
                    e_z = fmaf(f, nd.w, nd.z);
                    e_x = fmaf(g, hf.y, hf.x);
                    b_y = fmaf(g, hf.w, hf.z);
                    b_z = fmaf(g, hz.y, hz.x);
                } else {
                    const float(*sF)[WMAX] = sm.F;
                    e_y = (1.f - f) * sF[1][lb] + f * sF[1][lb + 1];
                    e_z = (1.f - f) * sF[2][lb] + f * sF[2][lb + 1];
                    e_x = (1.f - g) * sF[0][jb] + g * sF[0][jb + 1];
                    b_y = (1.f - g) * sF[3][jb] + g * sF[3][jb + 1];
                    b_z = (1.f - g) * sF[4][jb] + g * sF[4][jb + 1];
                }
                // --- Boris step for the Lorentz force (Bx = 0 in 1D)
                const float mx = px + hq * e_x, my = py + hq * e_y, mz = pz + hq * e_z;
                const float ig = rsqrt_ge1(1.f + mx * mx + my * my + mz * mz);
                const float ty = hq * b_y * ig, tz = hq * b_z * ig;
                const float sf = div_ge1(2.f, 1.f + ty * ty + tz * tz);
                const float sy = sf * ty, sz = sf * tz;
                const float ux = mx + my * tz - mz * ty;
                const float uy = my - mx * tz;
                const float uz = mz + mx * ty;
                const float lx = mx + uy * sz - uz * sy + hq * e_x;
                const float ly = my - ux * sz + hq * e_y;
                const float lz = mz + ux * sy + hq * e_z;
                float ign;  // 1 / gamma^{n+1/2}
                if (rr) {
                    // --- Eqs. (estim1, estimgamma): p(n) from p_L and p^{n-1/2}
                    const float bx_ = 0.5f * (lx + px), by_ = 0.5f * (ly + py), bz_ = 0.5f * (lz + pz);
                    const float igb = rsqrt_ge1(1.f + bx_ * bx_ + by_ * by_ + bz_ * bz_);
                    const float vx = bx_ * igb, vy = by_ * igb, vz = bz_ * igb;
                    // f_L = -(E + v x B)
                    const float fx = -(e_x + vy * b_z - vz * b_y);
                    const float fy = -(e_y - vx * b_z);
                    const float fz = -(e_z + vx * b_y);
                    const float av = vx * e_x + vy * e_y + vz * e_z;  // v.E = -v.f_L
                    // gamma^2 [f_L^2 - (v.E)^2] = f_L^2 + |p(n) x f_L|^2 (Lagrange identity),
                    // a sum of squares: no cancellation in single precision
                    const float cx = by_ * fz - bz_ * fy, cy = bz_ * fx - bx_ * fz, cz = bx_ * fy - by_ * fx;
                    const float br = fx * fx + fy * fy + fz * fz + cx * cx + cy * cy + cz * cz;
                    // Eq. (f_r) and Eq. (pertfull): p^{n+1/2} = p_L + dt f_R
                    const float kx = -eps * dt * (fy * b_z - fz * b_y - av * e_x + br * vx);
                    const float ky = -eps * dt * (-fx * b_z - av * e_y + br * vy);
                    const float kz = -eps * dt * (fx * b_y - av * e_z + br * vz);
                    px = lx + kx;
                    py = ly + ky;
                    pz = lz + kz;
                    // gamma(p_L) - gamma(p^{n+1/2}) without cancellation
                    const float qL = 1.f + lx * lx + ly * ly + lz * lz;
                    const float qN = 1.f + px * px + py * py + pz * pz;
                    ign = rsqrt_ge1(qN);
                    const float gL = qL * rsqrt_ge1(qL), gN = qN * ign;
                    rad -= div_ge1(kx * (lx + px) + ky * (ly + py) + kz * (lz + pz), gL + gN);
                } else {
                    px = lx;
                    py = ly;
                    pz = lz;
                    ign = rsqrt_ge1(1.f + px * px + py * py + pz * pz);
                }
                // --- move: x^{n+1} = x^n + dt p_x / gamma, in cell units
                const float vxn = px * ign;
                float fn = f + cfl * vxn;
                int d = fn >= 1.f ? 1 : (fn < 0.f ? -1 : 0);
                fn -= static_cast<float>(d);
                const bool edge = fn >= 1.f;  // rounded up to the boundary: same point as (c, 0)
                d = edge ? 0 : d;
                fn = edge ? 0.f : fn;
                int cnew = c + d, store_c = cnew;
                if (cnew < 0) {  // frozen at x = 0 (sorts under cell 0)
                    cnew = 0;
                    fn = 0.f;
                    d = 0;
                    store_c = -1;
                } else if (cnew >= Nx) {  // frozen at x = L (sorts under its last cell Nx-1)
                    cnew = Nx;
                    fn = 0.f;
                    store_c = -Nx;
                }
                // --- stencil record anchored at a = min(old bin, new bin): Jy, Jz on
                // nodes a..a+2 and Jx on half nodes a, a+1 (Esirkepov for linear shapes).
                // With x0, x1 the old and new positions measured from node a (both in
                // [0, 2)), the linear shape gives node a the weight max(0, 1 - x), node
                // a+2 max(0, x - 1) and node a+1 the rest; Jy and Jz take the weights
                // summed over the two positions (the time-averaged shape, doubled), Jx
                // the charge that crossed half nodes a and a+1.
                {
                    const bool up = d > 0, down = d < 0;
                    ka = down ? lb - 1 : lb;
                    const float x0 = down ? f + 1.f : f, x1 = up ? fn + 1.f : fn;
                    const float s0a = fmaxf(1.f - x0, 0.f), s0b = fmaxf(1.f - x1, 0.f);
                    const float s2a = fmaxf(x0 - 1.f, 0.f), s2b = fmaxf(x1 - 1.f, 0.f);
                    w0 = s0a + s0b;
                    w2 = s2a + s2b;
                    w1 = (2.f - w0) - w2;
                    const float hqi = hqw * ign;  // (q w / 2) / gamma in the window's units: ay = that times p_y
                    ay = hqi * py;
                    az = hqi * pz;
                    dj0 = s0a - s0b;
                    dj1 = s2b - s2a;
                }
                c = store_c;
                f = fn;
            }
            // merge the particle's record into this thread's running record; when
            // its anchor changes, the finished record is added: by the lane itself in
            // thin units and with 2 particles per thread (no warp vote per particle,
            // which lets the two particles' arithmetic overlap: 3-4 % faster on thin
            // plasma), through warp_add otherwise (4 per thread: the per-lane path
            // costs registers there, and dense foils rarely change anchor mid-round)
            const bool merge = ka < 0 || rk < 0 || ka == rk;
            if (thin || W == 2) {
                if (!merge) {
                    lane_add(rk, rv, sJ);
#pragma unroll
                    for (int q = 0; q < 8; ++q) rv[q] = 0.f;
                }
            } else if (__any_sync(FULL, !merge)) {
                warp_add(merge ? -1 : rk, rv, sJ);
                if (!merge) {
                    rk = -1;
#pragma unroll
                    for (int q = 0; q < 8; ++q) rv[q] = 0.f;
                }
            }
            if (ka >= 0) {  // the record's eight values, added to the running record
                rk = ka;
                rv[0] = fmaf(ay, w0, rv[0]);
                rv[1] = fmaf(ay, w1, rv[1]);
                rv[2] = fmaf(ay, w2, rv[2]);
                rv[3] = fmaf(az, w0, rv[3]);
                rv[4] = fmaf(az, w1, rv[4]);
                rv[5] = fmaf(az, w2, rv[5]);
                rv[6] = fmaf(jxf, dj0, rv[6]);
                rv[7] = fmaf(jxf, dj1, rv[7]);
            }
            act[j] = a;
            cn[j] = c;
            fo[j] = f;
            qx[j] = px;
            qy[j] = py;
            qz[j] = pz;
        }
        if (thin) {
            if (rk >= 0) lane_add(rk, rv, sJ);
        } else {
            warp_add(rk, rv, sJ);
        }
        rk = -1;
#pragma unroll
        for (int q = 0; q < 8; ++q) rv[q] = 0.f;
        // with 4 per thread (dense foils), a warp whose particles all stayed in
        // their cells leaves its cell slots as they are: a tenth of the written
        // bytes for most warps of a dense foil (the large run's push 0.440 ->
        // 0.425 ms); with 2 per thread (thin, hot plasma, where particles cross
        // cells every step) the vote cost more than it saved
        bool warp_moved = true;
        if constexpr (W == 4) {
            bool moved = false;
#pragma unroll
            for (int j = 0; j < W; ++j) moved = moved || cn[j] != comp(c4, j);
            warp_moved = __any_sync(FULL, moved);
        }
        if (slot_ok) {
            if (b4 >= start && b4 + W - 1 < end) {
                if (warp_moved) __stcs(reinterpret_cast<I*>(sp.cell + b4), Slot<W>::pack(cn));
                __stcs(reinterpret_cast<F*>(sp.off + b4), Slot<W>::pack(fo));
                __stcs(reinterpret_cast<F*>(sp.px + b4), Slot<W>::pack(qx));
                __stcs(reinterpret_cast<F*>(sp.py + b4), Slot<W>::pack(qy));
                __stcs(reinterpret_cast<F*>(sp.pz + b4), Slot<W>::pack(qz));
            } else {
#pragma unroll
                for (int j = 0; j < W; ++j) {
                    if (!act[j]) continue;
                    sp.cell[b4 + j] = cn[j];
                    sp.off[b4 + j] = fo[j];
                    sp.px[b4 + j] = qx[j];
                    sp.py[b4 + j] = qy[j];
                    sp.pz[b4 + j] = qz[j];
                }
            }
        }
    }



    // radiated energy of the unit: fixed-order warp reduction, warps summed in double
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rad += __shfl_xor_sync(FULL, rad, o);
    if (lane == 0) sred[warp] = static_cast<double>(rad);
    __syncthreads();  // also orders every shared-memory current update before the flush
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < PUSH_T / 32; ++w) t += sred[w];
        P.rad_part[u] += t * static_cast<double>(R.rad_w[s]);  // summed into the tally at the next flush
    }
    // flush the window: each exact sum shifted from record units to the
    // accumulators' 2^fp units (the run's fixed-point scale keeps it in range)
    for (int i = tid; i < L; i += PUSH_T) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long v = static_cast<long long>((static_cast<unsigned long long>(static_cast<unsigned>(sJ.hi[c][i])) << 32) | sJ.lo[c][i]);
            if (v) atomicAdd(R.J[par][c] + p0 + i, static_cast<unsigned long long>(v) << shift);
        }
    }
}

}  // namespace

void launch_push(const PushParams& P, int grid, int slot_w, cudaStream_t st) {
    if (grid <= 0) return;
    if (slot_w == 2)
        k_push_deposit<2><<<grid, PUSH_T, 0, st>>>(P);
    else
        k_push_deposit<4><<<grid, PUSH_T, 0, st>>>(P);
}

}  // namespace picrr
