// Spectrum entry point that allocates no device memory.
//
// pic_spectra keeps its integer bin counters in device memory that the
// handle allocates.  Some callers cannot allocate at the moment they want a
// spectrum: code that must not synchronise the device (cudaMalloc and
// cudaFree can), code running under a fixed memory budget owned by another
// allocator, or a plugin handed device buffers by a host application.  This
// file gives them pic_spectrum_noalloc: the same histogram, with its counters
// in one file-scope device array of this library.
//
// The array lives in every GPU that loads the library until the process
// exits.  All calls share it: each call clears the counters it uses before
// counting, so successive calls are independent, but calls whose work
// overlaps on the GPU (different streams, different threads) race on it.
#include <cmath>
#include <mutex>
#include <string>

#include "picrr.h"
#include "picrr_internal.cuh"

namespace picrr {
namespace {

// nbins counters + underflow + overflow
__device__ __align__(256) unsigned long long g_noalloc_bins[PIC_NOALLOC_MAX_BINS + 2];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned long long* g_bins_ptr[kMaxDevices] = {};


__global__ void k_noalloc_clear(unsigned long long* bins, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) bins[i] = 0ull;
}

__global__ void __launch_bounds__(256) k_noalloc_count(const float* px, const float* py, const float* pz,
                                                       int64_t n, double mass_mev, int nbins, double e_min,
                                                       double e_max, unsigned long long* bins) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const double x = px[i], y = py[i], z = pz[i];
        const double p2 = x * x + y * y + z * z;
        const double e = mass_mev * p2 / (sqrt(1.0 + p2) + 1.0);
        int k;
        if (e < e_min) {
            k = nbins;
        } else {
            const double kf = floor((e - e_min) / (e_max - e_min) * static_cast<double>(nbins));
            // written so that a NaN energy (never produced by a checked state) lands in the overflow
            k = kf < static_cast<double>(nbins) ? static_cast<int>(kf) : nbins + 1;
        }
        atomicAdd(&bins[k], 1ull);
    }
}

__global__ void k_noalloc_finish(const unsigned long long* bins, int nbins, double scale, double* counts) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nbins; i += gridDim.x * blockDim.x)
        counts[i] = static_cast<double>(bins[i]) * scale;
}

// Device address of the counter array on the current device (looked up once
// per device with that device current).
cudaError_t bins_address(int dev, unsigned long long** out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_bins_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_bins);
        if (e != cudaSuccess) return e;
        g_bins_ptr[dev] = static_cast<unsigned long long*>(p);
    }
    *out = g_bins_ptr[dev];
    return cudaSuccess;
}

pic_status noalloc_fail(pic_status st, const std::string& msg) {
    set_null_handle_error(msg);
    return st;
}

}  // namespace

}  // namespace picrr

extern "C" pic_status pic_spectrum_noalloc(const float* px, const float* py, const float* pz, int64_t n,
                                           double mass_me, double weight_dx, int nbins, double e_min_MeV,
                                           double e_max_MeV, double* counts, void* stream) {
    using namespace picrr;
    if (nbins < 1 || nbins > PIC_NOALLOC_MAX_BINS)
        return noalloc_fail(PIC_ERR_INVALID_ARG, "nbins must be in [1, " + std::to_string(PIC_NOALLOC_MAX_BINS) +
                                                     "] (the size of the library's fixed counter array)");
    if (n < 0 || (n > 0 && (!px || !py || !pz)) || !counts)
        return noalloc_fail(PIC_ERR_INVALID_ARG, "need n >= 0, device momenta for n > 0 and a device output");
    if (!(e_max_MeV > e_min_MeV) || !std::isfinite(e_min_MeV) || !std::isfinite(e_max_MeV) || !(mass_me > 0.0) ||
        !std::isfinite(weight_dx))
        return noalloc_fail(PIC_ERR_INVALID_ARG, "need e_max > e_min (finite), mass > 0, finite weight");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return noalloc_fail(PIC_ERR_CUDA, "no current CUDA device");
    }
    unsigned long long* bins = nullptr;
    e = bins_address(dev, &bins);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(PIC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nb2 = nbins + 2;
    k_noalloc_clear<<<(nb2 + 255) / 256, 256, 0, st>>>(bins, nb2);
    if (n > 0) {
        int64_t g = (n + 255) / 256;
        if (g > 1216) g = 1216;
        k_noalloc_count<<<static_cast<int>(g), 256, 0, st>>>(px, py, pz, n, mass_me * 0.51099895000, nbins,
                                                             e_min_MeV, e_max_MeV, bins);
    }
    const double width = (e_max_MeV - e_min_MeV) / nbins;
    k_noalloc_finish<<<(nbins + 255) / 256, 256, 0, st>>>(bins, nbins, weight_dx / width, counts);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(PIC_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return PIC_OK;
}
