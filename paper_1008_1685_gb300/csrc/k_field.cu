// 1D Yee update of one step, with the current of this step, total-field /
// scattered-field laser injection (incident values evaluated in double
// precision by the host for each step) and first-order Mur ends:
//   B^{n+1/2} = B^n - (dt/2) curl E^n,
//   E^{n+1}   = E^n + dt (curl B^{n+1/2} - J^{n+1/2}),
//   B^{n+1}   = B^{n+1/2} - (dt/2) curl E^{n+1}.
// Each block owns FIELD_NODES nodes of one run (a block table maps blocks to
// runs), FIELD_NODES / FIELD_T per thread, and recomputes the guard values it
// needs from its neighbours' old data, so one launch does the whole step
// (old and new fields live in separate buffers).  The block also converts
// the fixed-point current to float, zeroes the accumulators of the next
// step and adds the exact discrete Poynting flux through the two accounting
// planes.  (A version without shared memory and barriers, each thread
// recomputing the half-step B and new E it shares with its neighbours from
// global loads, ran at half the speed.)
#include "picrr_internal.cuh"

namespace picrr {

namespace {

// 64-bit fixed-point accumulator (2^fp units) to float from its two 32-bit
// halves (32-bit conversions only): hi * 2^(32-fp) + lo * 2^-fp.
__device__ __forceinline__ float fix_to_float(unsigned long long a, float lo_scale, float hi_scale) {
    const int hi = static_cast<int>(static_cast<long long>(a) >> 32);
    const unsigned lo = static_cast<unsigned>(a & 0xffffffffull);
    return fmaf(static_cast<float>(hi), hi_scale, static_cast<float>(lo) * lo_scale);
}

__global__ void __launch_bounds__(FIELD_T) k_field(const FieldParams P) {
    constexpr int T = FIELD_T, N = FIELD_NODES, K = N / T;
    // old E on nodes [i0-2, i0+N+1]; old B on half nodes [i0-2, i0+N], overwritten in place by
    // B^{n+1/2}; E^{n+1} on nodes [i0-1, i0+N]
    __shared__ float sEy[N + 4], sEz[N + 4], sBy[N + 3], sBz[N + 3];
    __shared__ float nEy[N + 2], nEz[N + 2];
    const int tid = threadIdx.x;
    const int run = P.blk_run[blockIdx.x];
    const RunDev& R = P.runs[run];
    if (!R.active) return;  // block-uniform
    const int i0 = P.blk_i0[blockIdx.x];
    const int Nx = R.Nx, is = R.is, glen = R.glen;
    const int par = static_cast<int>((P.gstep + R.fpar) & 1);
    const float* const* Fo = R.F[par];
    float* const* Fn = R.F[1 - par];
    const unsigned long long* const* Jacc = R.J[par];
    unsigned long long* const* Jnext = R.J[1 - par];
    const float* inc = P.inc + 6 * run;
    const float c = P.c, hc = P.hc, fdt = P.fdt, fpi = R.fp_inv, fph = R.fp_inv * 4294967296.0f;

    // Every load of the block is issued here, before the first barrier: the old fields and the
    // transverse current of the stencil (J on node i0-1+q kept in the register of the thread that
    // updates E there), and Ex and Jx of the owned nodes.
    unsigned long long jy[K + 1], jz[K + 1], jx[K];
    float ex[K];
#pragma unroll
    for (int k = 0; k <= K; ++k) {
        const int q = tid + k * T;
        if (k == K && q >= N + 4) break;  // the 4 guard entries past the tile
        const int i = i0 - 2 + q + PADF;  // padded index, >= PADF - 2 >= 0
        const bool in = i < glen;         // the last block reaches past the array end
        sEy[q] = in ? Fo[1][i] : 0.f;
        sEz[q] = in ? Fo[2][i] : 0.f;
        if (q < N + 3) {
            sBy[q] = in ? Fo[3][i] : 0.f;
            sBz[q] = in ? Fo[4][i] : 0.f;
        }
        // J on node i0-1+q for q < N+2 (one further than the old fields: index i+1)
        const bool jin = q < N + 2 && i + 1 < glen;
        jy[k] = jin ? Jacc[1][i + 1] : 0ull;
        jz[k] = jin ? Jacc[2][i + 1] : 0ull;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int pi = i0 + tid + k * T + PADF;
        const bool own = i0 + tid + k * T < Nx;
        jx[k] = own ? Jacc[0][pi] : 0ull;
        ex[k] = own ? Fo[0][pi] : 0.f;
    }
    __syncthreads();

    // B^{n+1/2} on half nodes j = i0-2+q, in place (entry q is read and written by one thread only)
#pragma unroll
    for (int k = 0; k <= K; ++k) {
        const int q = tid + k * T;
        if (k == K && q >= N + 3) break;
        const int j = i0 - 2 + q;
        float by = sBy[q] + hc * (sEz[q + 1] - sEz[q]);
        float bz = sBz[q] - hc * (sEy[q + 1] - sEy[q]);
        if (j == is - 1) {  // scattered side of the source plane: remove the incident E at t_n
            bz += hc * inc[0];
            by -= hc * inc[1];
        }
        sBy[q] = by;
        sBz[q] = bz;
    }
    __syncthreads();

    // E^{n+1} on nodes i = i0-1+q (interior formula; Mur nodes below)
#pragma unroll
    for (int k = 0; k <= K; ++k) {
        const int q = tid + k * T;
        if (k == K && q >= N + 2) break;
        const int i = i0 - 1 + q;
        // node i: old E at sE[q+1], half nodes i-1, i at sB[q], sB[q+1]
        float ey = sEy[q + 1] - c * (sBz[q + 1] - sBz[q]) - fdt * fix_to_float(jy[k], fpi, fph);
        float ez = sEz[q + 1] + c * (sBy[q + 1] - sBy[q]) - fdt * fix_to_float(jz[k], fpi, fph);
        if (i == is) {  // total side: add the incident B at half node is-1/2, time t_n + dt/2
            ey += c * inc[2];
            ez += c * inc[3];
        }
        if (i < 1 || i > Nx - 1) {
            ey = 0.f;
            ez = 0.f;
        }
        nEy[q] = ey;
        nEz[q] = ez;
    }
    __syncthreads();
    // first-order Mur ends: E_0 = E_1^n + km (E_1^{n+1} - E_0^n), same at Nx
    if (tid == 0) {
        const float km = (c - 1.f) / (c + 1.f);
        if (i0 - 1 <= 0 && 0 <= i0 + N) {
            const int q = 0 - (i0 - 1);
            // node 0: old at sE[q+1], node 1 old at sE[q+2], new node 1 at nE[q+1]
            nEy[q] = sEy[q + 2] + km * (nEy[q + 1] - sEy[q + 1]);
            nEz[q] = sEz[q + 2] + km * (nEz[q + 1] - sEz[q + 1]);
        }
        if (i0 - 1 <= Nx && Nx <= i0 + N) {
            const int q = Nx - (i0 - 1);
            nEy[q] = sEy[q] + km * (nEy[q - 1] - sEy[q + 1]);
            nEz[q] = sEz[q] + km * (nEz[q - 1] - sEz[q + 1]);
        }
    }
    __syncthreads();

    // owned outputs: node / half node i = i0 + q
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int q = tid + k * T;  // node i: nE[q+1], sE[q+2]; half node i: sB[q+2]
        const int i = i0 + q;
        const int pi = i + PADF;
        if (i <= Nx) {
            Fn[1][pi] = nEy[q + 1];
            Fn[2][pi] = nEz[q + 1];
        }
        if (i < Nx) {
            float by = sBy[q + 2] + hc * (nEz[q + 2] - nEz[q + 1]);
            float bz = sBz[q + 2] - hc * (nEy[q + 2] - nEy[q + 1]);
            if (i == is - 1) {  // incident E at t_{n+1}
                bz += hc * inc[4];
                by -= hc * inc[5];
            }
            Fn[3][pi] = by;
            Fn[4][pi] = bz;
            Fn[0][pi] = ex[k] - fdt * fix_to_float(jx[k], fpi, fph);
        }
        // exact discrete Poynting flux through the accounting planes
        const int a = is + 1, b = Nx - 1;
        if (i == a) {
            const double ey = 0.5 * (static_cast<double>(sEy[q + 2]) + nEy[q + 1]);
            const double ez = 0.5 * (static_cast<double>(sEz[q + 2]) + nEz[q + 1]);
            R.tally[1] += P.dt * (ey * sBz[q + 1] - ez * sBy[q + 1]);
        }
        if (i == b) {
            const double ey = 0.5 * (static_cast<double>(sEy[q + 2]) + nEy[q + 1]);
            const double ez = 0.5 * (static_cast<double>(sEz[q + 2]) + nEz[q + 1]);
            R.tally[2] += P.dt * (ey * sBz[q + 2] - ez * sBy[q + 2]);
        }
    }
    // zero the accumulators of the next step: owned padded range of this block
    {
        const int lo = (i0 == 0) ? 0 : i0 + PADF;
        const int hi = (i0 + N > Nx) ? Nx + 2 * PADF + 1 : i0 + N + PADF;
        for (int pi = lo + tid; pi < hi; pi += T) {
            Jnext[0][pi] = 0ull;
            Jnext[1][pi] = 0ull;
            Jnext[2][pi] = 0ull;
        }
    }
}

}  // namespace

void launch_field(const FieldParams& P, int grid, cudaStream_t st) {
    k_field<<<grid, FIELD_T, 0, st>>>(P);
}

}  // namespace picrr
