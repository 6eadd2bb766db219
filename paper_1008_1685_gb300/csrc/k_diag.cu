// Diagnostics: field and kinetic energy (FP64 accumulation, fixed-order
// reductions so repeated calls give identical bits), the kinetic-energy
// spectrum (integer bin counts), and the skin-layer snapshot of Sec. 4: the
// friction coefficient d of Eq. (damping) and the quantum parameter chi of
// the classical validity condition (Sec. 2) for every particle.
#include "picrr_internal.cuh"

namespace picrr {

namespace {

constexpr int DIAG_T = 256;

__device__ __forceinline__ double block_sum(double v, double* sred) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < DIAG_T / 32; ++w) t += sred[w];
    return t;
}

// Field energy of the accounting region at integer time n: nodes
// [is+1, Nx-1] carry (Ey^2 + Ez^2)/2; half nodes [is+1, Nx-2] carry
// (B^{n-1/2}.B^{n+1/2})/2 = ((B^n)^2 - ((dt/2) curl E^n)^2)/2; all half nodes
// carry Ex^2/2.  Times dx on the host.
__global__ void __launch_bounds__(DIAG_T) k_field_energy(const DiagParams D, double* partials) {
    __shared__ double sred[DIAG_T / 32];
    const int a = D.is + 1, b = D.Nx - 1;
    double w = 0.0;
    for (int i = blockIdx.x * DIAG_T + threadIdx.x; i <= D.Nx; i += gridDim.x * DIAG_T) {
        const int p = i + PADF;
        if (i >= a && i <= b) {
            const double ey = D.F[1][p], ez = D.F[2][p];
            w += 0.5 * (ey * ey + ez * ez);
        }
        if (i >= a && i <= b - 1) {
            const double by = D.F[3][p], bz = D.F[4][p];
            const double dy = static_cast<double>(D.hc) * (static_cast<double>(D.F[2][p + 1]) - D.F[2][p]);
            const double dz = static_cast<double>(D.hc) * (static_cast<double>(D.F[1][p + 1]) - D.F[1][p]);
            w += 0.5 * (by * by - dy * dy + bz * bz - dz * dz);
        }
        if (i < D.Nx) {
            const double ex = D.F[0][p];
            w += 0.5 * ex * ex;
        }
    }
    const double t = block_sum(w, sred);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// Sum of (gamma - 1) over all particles of a species (frozen ones included).
__global__ void __launch_bounds__(DIAG_T) k_kinetic(DevSpecies sp, int64_t n, double* partials) {
    __shared__ double sred[DIAG_T / 32];
    double w = 0.0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * DIAG_T + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * DIAG_T) {
        const double px = sp.px[i], py = sp.py[i], pz = sp.pz[i];
        const double p2 = px * px + py * py + pz * pz;
        w += p2 / (sqrt(1.0 + p2) + 1.0);
    }
    const double t = block_sum(w, sred);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void __launch_bounds__(1024) k_reduce(const double* partials, int n, double scale, double* out) {
    __shared__ double sred[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += 1024) v += partials[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 32; ++w) t += sred[w];
        *out = t * scale;
    }
}

// bins[0..nbins) counts, bins[nbins] underflow, bins[nbins+1] overflow.
// Energy m c^2 (gamma - 1) in MeV evaluated in double.
__global__ void __launch_bounds__(DIAG_T) k_spectrum(DevSpecies sp, int64_t n, double mass_mev, int nbins,
                                                     double e_min, double e_max, unsigned long long* bins) {
    extern __shared__ unsigned int sh[];
    const bool use_sh = nbins + 2 <= 8192;
    if (use_sh)
        for (int i = threadIdx.x; i < nbins + 2; i += DIAG_T) sh[i] = 0u;
    __syncthreads();
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * DIAG_T + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * DIAG_T) {
        const double px = sp.px[i], py = sp.py[i], pz = sp.pz[i];
        const double p2 = px * px + py * py + pz * pz;
        const double e = mass_mev * p2 / (sqrt(1.0 + p2) + 1.0);
        int k;
        if (e < e_min) {
            k = nbins;
        } else {
            const double kf = floor((e - e_min) / (e_max - e_min) * static_cast<double>(nbins));
            // written so that a NaN energy (never produced by a checked state) lands in the overflow
            k = kf < static_cast<double>(nbins) ? static_cast<int>(kf) : nbins + 1;
        }
        if (use_sh) atomicAdd(&sh[k], 1u);
        else atomicAdd(&bins[k], 1ull);
    }
    __syncthreads();
    if (use_sh)
        for (int i = threadIdx.x; i < nbins + 2; i += DIAG_T)
            if (sh[i]) atomicAdd(&bins[i], static_cast<unsigned long long>(sh[i]));
}

// One thread per particle.  Linear gather as in the push (nodes for Ey, Ez;
// half nodes for Ex, By, Bz; zero guard elements beyond the grid), then
// gamma^2 [f_L^2 - (v.f_L)^2] as the sum of squares f_L^2 + |p x f_L|^2
// (Lagrange identity with p = gamma v).
__global__ void __launch_bounds__(DIAG_T) k_snapshot(DevSpecies sp, int64_t n, const SnapParams S, float* d_out,
                                                     float* chi_out, unsigned long long* out) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * DIAG_T + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * DIAG_T) {
        const int c = sp.cell[i];
        float d = 0.f, chi = 0.f;
        if (c >= 0) {  // frozen particles (c < 0) feel no field
            const float f = sp.off[i];
            const int q = c + PADF;
            const float e_y = (1.f - f) * S.F[1][q] + f * S.F[1][q + 1];
            const float e_z = (1.f - f) * S.F[2][q] + f * S.F[2][q + 1];
            const float h = f - 0.5f;
            const int jb = h < 0.f ? q - 1 : q;
            const float g = h < 0.f ? h + 1.f : h;
            const float e_x = (1.f - g) * S.F[0][jb] + g * S.F[0][jb + 1];
            const float b_y = (1.f - g) * S.F[3][jb] + g * S.F[3][jb + 1];
            const float b_z = (1.f - g) * S.F[4][jb] + g * S.F[4][jb + 1];
            const float px = sp.px[i], py = sp.py[i], pz = sp.pz[i];
            const float ig = rsqrtf(1.f + px * px + py * py + pz * pz);
            const float vx = px * ig, vy = py * ig, vz = pz * ig;
            const float fx = -(e_x + vy * b_z - vz * b_y);
            const float fy = -(e_y - vx * b_z);
            const float fz = -(e_z + vx * b_y);
            const float cx = py * fz - pz * fy, cy = pz * fx - px * fz, cz = px * fy - py * fx;
            const float br = fx * fx + fy * fy + fz * fz + cx * cx + cy * cy + cz * cz;
            d = S.eps * br;
            chi = sqrtf(br) * S.ecr_inv;
        }
        if (d_out) d_out[i] = d;
        if (chi_out) chi_out[i] = chi;
        // maxima of non-negative floats through their bit patterns; integer count
        atomicMax(reinterpret_cast<unsigned int*>(&out[0]), __float_as_uint(d));
        atomicMax(reinterpret_cast<unsigned int*>(&out[1]), __float_as_uint(chi));
        const unsigned flagged = __ballot_sync(__activemask(), chi >= S.chi_flag);
        if (flagged && (threadIdx.x & 31) == __ffs(__activemask()) - 1)
            atomicAdd(&out[2], static_cast<unsigned long long>(__popc(flagged)));
    }
}

// Checks of an uploaded particle array: out[0] counts cells outside [0, Nx),
// out[1] offsets outside [0, 1) or non-finite momenta, out[2] places where the
// cells decrease (the array is not in cell order).
__global__ void __launch_bounds__(DIAG_T) k_validate(const int32_t* cell, const float* off, const float* px,
                                                     const float* py, const float* pz, int64_t n, int Nx,
                                                     unsigned long long* out) {
    unsigned long long bad_cell = 0, bad_val = 0, down = 0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * DIAG_T + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * DIAG_T) {
        const int c = cell[i];
        const float f = off[i];
        bad_cell += (c < 0 || c >= Nx) ? 1 : 0;
        bad_val += (!(f >= 0.f && f < 1.f) || !isfinite(px[i]) || !isfinite(py[i]) || !isfinite(pz[i])) ? 1 : 0;
        down += (i > 0 && c < cell[i - 1]) ? 1 : 0;
    }
    if (bad_cell) atomicAdd(&out[0], bad_cell);
    if (bad_val) atomicAdd(&out[1], bad_val);
    if (down) atomicAdd(&out[2], down);
}

// Self-test of the bounded device wait: an mbarrier that expects two
// arrivals gets one, so its phase never completes; the wait (the helper the
// push kernel uses for its field window) gives up after its bounded number of
// polls and the kernel records the timeout in the status word.
__global__ void k_wait_selftest(int* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 2);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_arrive(&bar);
    const bool got = mbar_wait_bounded(&bar, 0);
    if (!__syncthreads_and(got) && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
}

}  // namespace

void launch_wait_selftest(int* status, cudaStream_t st) { k_wait_selftest<<<1, 32, 0, st>>>(status); }

void launch_validate(const int32_t* cell, const float* off, const float* px, const float* py, const float* pz,
                     int64_t n, int Nx, unsigned long long* out, cudaStream_t st) {
    int64_t g = (n + DIAG_T - 1) / DIAG_T;
    if (g > 4864) g = 4864;
    if (g < 1) g = 1;
    k_validate<<<static_cast<int>(g), DIAG_T, 0, st>>>(cell, off, px, py, pz, n, Nx, out);
}

void launch_snapshot(DevSpecies sp, int64_t n, const SnapParams& S, float* d_out, float* chi_out,
                     unsigned long long* out, cudaStream_t st) {
    int64_t g = (n + DIAG_T - 1) / DIAG_T;
    if (g > 4864) g = 4864;
    if (g < 1) g = 1;
    k_snapshot<<<static_cast<int>(g), DIAG_T, 0, st>>>(sp, n, S, d_out, chi_out, out);
}

int launch_field_energy(const DiagParams& D, double* partials, int max_blocks, cudaStream_t st) {
    int g = (D.Nx + 1 + DIAG_T - 1) / DIAG_T;
    if (g > max_blocks) g = max_blocks;
    if (g < 1) g = 1;
    k_field_energy<<<g, DIAG_T, 0, st>>>(D, partials);
    return g;
}

int launch_kinetic(DevSpecies sp, int64_t n, double* partials, int max_blocks, cudaStream_t st) {
    int64_t g = (n + DIAG_T - 1) / DIAG_T;
    if (g > max_blocks) g = max_blocks;
    if (g < 1) g = 1;
    k_kinetic<<<static_cast<int>(g), DIAG_T, 0, st>>>(sp, n, partials);
    return static_cast<int>(g);
}

void launch_reduce_partials(const double* partials, int n, double scale, double* out, cudaStream_t st) {
    k_reduce<<<1, 1024, 0, st>>>(partials, n, scale, out);
}

void launch_spectrum(DevSpecies sp, int64_t n, double mass_mev, int nbins, double e_min, double e_max,
                     unsigned long long* bins, cudaStream_t st) {
    int64_t g = (n + DIAG_T - 1) / DIAG_T;
    if (g > 1216) g = 1216;
    if (g < 1) g = 1;
    const size_t sh = (nbins + 2 <= 8192) ? sizeof(unsigned int) * (nbins + 2) : 0;
    k_spectrum<<<static_cast<int>(g), DIAG_T, sh, st>>>(sp, n, mass_mev, nbins, e_min, e_max, bins);
}

}  // namespace picrr
