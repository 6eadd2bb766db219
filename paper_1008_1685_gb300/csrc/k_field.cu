// 1D Yee update of one step, with the current of this step, total-field /
// scattered-field laser injection and first-order Mur ends:
//   B^{n+1/2} = B^n - (dt/2) curl E^n,
//   E^{n+1}   = E^n + dt (curl B^{n+1/2} - J^{n+1/2}),
//   B^{n+1}   = B^{n+1/2} - (dt/2) curl E^{n+1}.
// Each block owns FIELD_T nodes and recomputes the two guard values it
// needs from its neighbours' old data, so one launch does the whole step
// (old and new fields live in separate buffers).  The block also converts
// the fixed-point current to float, zeroes the accumulators of the next
// step, adds the exact discrete Poynting flux through the two accounting
// planes, and (block 0) sums the radiated energy of the push kernel's units
// in a fixed order.
#include "picrr_internal.cuh"

namespace picrr {

namespace {

constexpr double kPi = 3.14159265358979323846;

// Incident field at retarded time t (double precision phase and envelope):
// Ey_inc = Bz_inc = ay, Ez_inc = -By_inc = az.
__device__ void incident(const LaserParams& L, double t, float* ay, float* az) {
    *ay = 0.f;
    *az = 0.f;
    if (!L.on || t < 0.0 || t > L.tau) return;
    double g;
    if (L.env == 0) {
        const double q = sin(kPi * t / L.tau);
        g = q * q;
    } else if (t < L.rise) {
        const double q = sin(0.5 * kPi * t / L.rise);
        g = q * q;
    } else if (t > L.tau - L.rise) {
        const double q = sin(0.5 * kPi * (L.tau - t) / L.rise);
        g = q * q;
    } else {
        g = 1.0;
    }
    double sn, cs;
    sincos(t, &sn, &cs);
    if (L.pol == 0) {
        *ay = static_cast<float>(L.a0 * g * sn);
    } else {
        const double a = L.a0 * 0.70710678118654752440;
        *ay = static_cast<float>(a * g * sn);
        *az = static_cast<float>(-a * g * cs);
    }
}

__global__ void __launch_bounds__(FIELD_T) k_field(const FieldParams P) {
    constexpr int T = FIELD_T;
    // old E on nodes [i0-2, i0+T+1], old B and Ex on half nodes [i0-2, i0+T]
    __shared__ float sEy[T + 4], sEz[T + 4], sBy[T + 3], sBz[T + 3];
    __shared__ float hBy[T + 3], hBz[T + 3];  // B^{n+1/2} on half nodes [i0-2, i0+T]
    __shared__ float nEy[T + 2], nEz[T + 2];  // E^{n+1} on nodes [i0-1, i0+T]
    __shared__ float sJy[T + 2], sJz[T + 2];  // J on nodes [i0-1, i0+T]
    __shared__ double sred[32];

    const int tid = threadIdx.x;
    const int i0 = blockIdx.x * T;
    const int Nx = P.Nx, is = P.is;
    const float c = P.c, hc = P.hc, fdt = P.fdt, fpi = P.fp_inv;

    for (int q = tid; q < T + 4; q += T) {
        const int i = i0 - 2 + q + PADF;  // padded index, >= PADF - 2 >= 0
        const bool in = i < P.glen;       // the last block reaches past the array end
        sEy[q] = in ? P.Fo[1][i] : 0.f;
        sEz[q] = in ? P.Fo[2][i] : 0.f;
        if (q < T + 3) {
            sBy[q] = in ? P.Fo[3][i] : 0.f;
            sBz[q] = in ? P.Fo[4][i] : 0.f;
        }
        if (q >= 1 && q < T + 3) {  // J on nodes [i0-1, i0+T]
            sJy[q - 1] = in ? __ll2float_rn(static_cast<long long>(P.Jacc[1][i])) * fpi : 0.f;
            sJz[q - 1] = in ? __ll2float_rn(static_cast<long long>(P.Jacc[2][i])) * fpi : 0.f;
        }
    }
    __syncthreads();

    const double tn = static_cast<double>(P.n) * P.dt;
    // B^{n+1/2} on half nodes j = i0-2+q
    for (int q = tid; q < T + 3; q += T) {
        const int j = i0 - 2 + q;
        float by = sBy[q] + hc * (sEz[q + 1] - sEz[q]);
        float bz = sBz[q] - hc * (sEy[q + 1] - sEy[q]);
        if (j == is - 1 && P.laser.on) {  // scattered side of the source plane: remove the incident E
            float ay, az;
            incident(P.laser, tn, &ay, &az);
            bz += hc * ay;
            by -= hc * az;
        }
        hBy[q] = by;
        hBz[q] = bz;
    }
    __syncthreads();

    // E^{n+1} on nodes i = i0-1+q (interior formula; Mur nodes below)
    for (int q = tid; q < T + 2; q += T) {
        const int i = i0 - 1 + q;
        // node i: old E at sE[q+1], half nodes i-1, i at hB[q], hB[q+1]
        float ey = sEy[q + 1] - c * (hBz[q + 1] - hBz[q]) - fdt * sJy[q];
        float ez = sEz[q + 1] + c * (hBy[q + 1] - hBy[q]) - fdt * sJz[q];
        if (i == is && P.laser.on) {  // total side: add the incident B at half node is-1/2
            float ay, az;
            incident(P.laser, tn + 0.5 * P.dt + 0.5 * P.dx, &ay, &az);
            ey += c * ay;
            ez += c * az;
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
        if (i0 - 1 <= 0 && 0 <= i0 + T) {
            const int q = 0 - (i0 - 1);
            // node 0: old at sE[q+1], node 1 old at sE[q+2], new node 1 at nE[q+1]
            nEy[q] = sEy[q + 2] + km * (nEy[q + 1] - sEy[q + 1]);
            nEz[q] = sEz[q + 2] + km * (nEz[q + 1] - sEz[q + 1]);
        }
        if (i0 - 1 <= Nx && Nx <= i0 + T) {
            const int q = Nx - (i0 - 1);
            nEy[q] = sEy[q] + km * (nEy[q - 1] - sEy[q + 1]);
            nEz[q] = sEz[q] + km * (nEz[q - 1] - sEz[q + 1]);
        }
    }
    __syncthreads();

    // owned outputs: node / half node i = i0 + tid
    {
        const int i = i0 + tid;
        const int q = tid;  // node i: nE[q+1], sE[q+2]; half node i: hB[q+2]
        const int pi = i + PADF;
        if (i <= Nx) {
            P.Fn[1][pi] = nEy[q + 1];
            P.Fn[2][pi] = nEz[q + 1];
            P.Jf[1][pi] = sJy[q + 1];
            P.Jf[2][pi] = sJz[q + 1];
        }
        if (i < Nx) {
            float by = hBy[q + 2] + hc * (nEz[q + 2] - nEz[q + 1]);
            float bz = hBz[q + 2] - hc * (nEy[q + 2] - nEy[q + 1]);
            if (i == is - 1 && P.laser.on) {
                float ay, az;
                incident(P.laser, tn + P.dt, &ay, &az);
                bz += hc * ay;
                by -= hc * az;
            }
            P.Fn[3][pi] = by;
            P.Fn[4][pi] = bz;
            const float jx = __ll2float_rn(static_cast<long long>(P.Jacc[0][pi])) * fpi;
            P.Jf[0][pi] = jx;
            P.Fn[0][pi] = P.Fo[0][pi] - fdt * jx;
        }
        // exact discrete Poynting flux through the accounting planes
        const int a = is + 1, b = Nx - 1;
        if (i == a) {
            const double ey = 0.5 * (static_cast<double>(sEy[q + 2]) + nEy[q + 1]);
            const double ez = 0.5 * (static_cast<double>(sEz[q + 2]) + nEz[q + 1]);
            P.tally[1] += P.dt * (ey * hBz[q + 1] - ez * hBy[q + 1]);
        }
        if (i == b) {
            const double ey = 0.5 * (static_cast<double>(sEy[q + 2]) + nEy[q + 1]);
            const double ez = 0.5 * (static_cast<double>(sEz[q + 2]) + nEz[q + 1]);
            P.tally[2] += P.dt * (ey * hBz[q + 2] - ez * hBy[q + 2]);
        }
    }
    // zero the accumulators of the next step: owned padded range of this block
    {
        const int lo = (blockIdx.x == 0) ? 0 : i0 + PADF;
        const int hi = (i0 + T > Nx) ? Nx + 2 * PADF + 1 : i0 + T + PADF;
        for (int pi = lo + tid; pi < hi; pi += T) {
            P.Jnext[0][pi] = 0ull;
            P.Jnext[1][pi] = 0ull;
            P.Jnext[2][pi] = 0ull;
        }
    }
    // block 0: radiated energy of this step, fixed summation order
    if (blockIdx.x == 0) {
        const int nu = P.nunits[0];
        double acc = 0.0;
        for (int u = tid; u < nu; u += T) acc += P.rad_part[u];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((tid & 31) == 0) sred[tid >> 5] = acc;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < T / 32; ++w) t += sred[w];
            P.tally[0] += t;
        }
    }
}

}  // namespace

void launch_field(const FieldParams& P, int grid, cudaStream_t st) {
    k_field<<<grid, FIELD_T, 0, st>>>(P);
}

}  // namespace picrr
