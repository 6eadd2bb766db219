// Single electrons in analytic plane waves, many at once: the paper's
// validation path (Sec. 3), batched over scans of amplitude and initial
// momentum.  One thread integrates one electron in double precision (a
// reference integrator, not the PIC hot path):
//   - the leapfrog pusher of Sec. 3: Boris rotation for the Lorentz force plus
//     the RR kick of Eqs. (f_r, pertfull, estim1, estimgamma), fields at
//     (t_n, x^n), then x^{n+1} = x^n + dt v_x^{n+1/2};
//   - classical RK4 on the lab-frame LL equation, Eq. (3dLL), with or without
//     its field-derivative term.
// Plane waves travel along +x with phase phi = t - x and B = x_hat x E:
//   wave 0: LP, Ey = a0 cos(phi);
//   wave 1: CP, (Ey, Ez) = (a0/sqrt2)(cos(phi), sin(phi));
//   wave 2: LP pulse, Ey = a0 sin^2(pi phi/tau) cos(phi) for 0 <= phi <= tau.
#include <string>

#include "picrr.h"
#include "picrr_internal.cuh"

namespace picrr {

namespace {

constexpr int ELEC_T = 128;
constexpr double kPiD = 3.14159265358979323846;

struct Wave {
    int kind;
    double a0, tau;
};

// E(phi) and dE/dphi (x component zero); B = (0, -Ez, Ey).
__device__ void wave_at(const Wave& w, double phi, double& ey, double& ez, double& dey, double& dez) {
    ey = ez = dey = dez = 0.0;
    double s, c;
    sincos(phi, &s, &c);
    if (w.kind == 0) {
        ey = w.a0 * c;
        dey = -w.a0 * s;
    } else if (w.kind == 1) {
        const double a = w.a0 * 0.70710678118654752440;
        ey = a * c;
        ez = a * s;
        dey = -a * s;
        dez = a * c;
    } else if (phi >= 0.0 && phi <= w.tau) {
        double se, ce;
        sincos(kPiD * phi / w.tau, &se, &ce);
        const double g = se * se, dg = 2.0 * se * ce * kPiD / w.tau;
        ey = w.a0 * g * c;
        dey = w.a0 * (dg * c - g * s);
    }
}

// Lab-frame LL force of Eq. (3dLL) on an electron (charge -1) with momentum p
// in the wave at phase phi.
__device__ void ll_force(const Wave& w, double phi, const double p[3], double eps, bool rr, bool deriv,
                         double f[3], double* vx_out) {
    const double g = sqrt(1.0 + p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    const double vx = p[0] / g, vy = p[1] / g, vz = p[2] / g;
    double ey, ez, dey, dez;
    wave_at(w, phi, ey, ez, dey, dez);
    const double by = -ez, bz = ey;
    // L = E + v x B (Bx = 0, Ex = 0)
    const double lx = vy * bz - vz * by, ly = ey - vx * bz, lz = ez + vx * by;
    f[0] = -lx;
    f[1] = -ly;
    f[2] = -lz;
    if (rr) {
        const double vE = vy * ey + vz * ez;
        // (E + v x B) x B + (v.E) E
        const double tx = ly * bz - lz * by, ty = -lx * bz, tz = lx * by;
        const double sq = g * g * (lx * lx + ly * ly + lz * lz - vE * vE);
        f[0] += eps * (tx - sq * vx);
        f[1] += eps * (ty + vE * ey - sq * vy);
        f[2] += eps * (tz + vE * ez - sq * vz);
        if (deriv) {
            // (d/dt + v.grad) of a field of t - x is (1 - v_x) d/dphi; dB = (0, -dEz, dEy)
            const double k = eps * g * (1.0 - vx);
            const double dby = -dez, dbz = dey;
            f[0] -= k * (vy * dbz - vz * dby);
            f[1] -= k * (dey - vx * dbz);
            f[2] -= k * (dez + vx * dby);
        }
    }
    *vx_out = vx;
}

__global__ void __launch_bounds__(ELEC_T) k_electron_rk4(const pic_electron_case* cases, int64_t n, double dt,
                                                          int64_t nsteps, int every, double eps, int flags,
                                                          double* out, int64_t nsamples) {
    const int64_t c = static_cast<int64_t>(blockIdx.x) * ELEC_T + threadIdx.x;
    if (c >= n) return;
    const pic_electron_case C = cases[c];
    const Wave w{C.wave, C.a0, C.tau};
    const bool rr = flags & 1, deriv = (flags & 2) != 0;
    double x = C.x0, p[3] = {C.p0[0], C.p0[1], C.p0[2]};
    int64_t k = 0;
    for (int64_t s = 0; s < nsteps; ++s) {
        const double t = static_cast<double>(s) * dt;
        double f1[3], f2[3], f3[3], f4[3], v1, v2, v3, v4, q[3];
        ll_force(w, t - x, p, eps, rr, deriv, f1, &v1);
        for (int i = 0; i < 3; ++i) q[i] = p[i] + 0.5 * dt * f1[i];
        ll_force(w, t + 0.5 * dt - (x + 0.5 * dt * v1), q, eps, rr, deriv, f2, &v2);
        for (int i = 0; i < 3; ++i) q[i] = p[i] + 0.5 * dt * f2[i];
        ll_force(w, t + 0.5 * dt - (x + 0.5 * dt * v2), q, eps, rr, deriv, f3, &v3);
        for (int i = 0; i < 3; ++i) q[i] = p[i] + dt * f3[i];
        ll_force(w, t + dt - (x + dt * v3), q, eps, rr, deriv, f4, &v4);
        x += dt / 6.0 * (v1 + 2.0 * v2 + 2.0 * v3 + v4);
        for (int i = 0; i < 3; ++i) p[i] += dt / 6.0 * (f1[i] + 2.0 * f2[i] + 2.0 * f3[i] + f4[i]);
        if ((s + 1) % every == 0 && k < nsamples) {
            double* o = out + (c * nsamples + k++) * 5;
            o[0] = static_cast<double>(s + 1) * dt;
            o[1] = x;
            o[2] = p[0];
            o[3] = p[1];
            o[4] = p[2];
        }
    }
}

// One step of the pusher of Sec. 3 for an electron: p holds p^{n-1/2} on
// entry and p^{n+1/2} on return; E = (0, ey, ez), B = (0, -ez, ey) at t_n, x^n.
__device__ void leapfrog_kick(double p[3], double ey, double ez, double dt, double eps, bool rr) {
    const double by = -ez, bz = ey;
    const double h = -0.5 * dt;  // q/m (dt/2) for an electron
    // Boris: half E kick, rotation about B, half E kick
    const double mx = p[0], my = p[1] + h * ey, mz = p[2] + h * ez;
    const double gm = sqrt(1.0 + mx * mx + my * my + mz * mz);
    const double ty = h * by / gm, tz = h * bz / gm;
    const double s = 2.0 / (1.0 + ty * ty + tz * tz);
    // m' = m + m x t ; m+ = m + m' x (s t)
    const double ux = mx + (my * tz - mz * ty), uy = my - mx * tz, uz = mz + mx * ty;
    const double lx = mx + s * (uy * tz - uz * ty), ly = my - s * ux * tz, lz = mz + s * ux * ty;
    const double pLx = lx, pLy = ly + h * ey, pLz = lz + h * ez;
    if (!rr) {
        p[0] = pLx;
        p[1] = pLy;
        p[2] = pLz;
        return;
    }
    // Eq. (estim1): p(n) = (p_L^{n+1/2} + p^{n-1/2}) / 2; Eq. (estimgamma): gamma(n) from it
    const double qx = 0.5 * (pLx + p[0]), qy = 0.5 * (pLy + p[1]), qz = 0.5 * (pLz + p[2]);
    const double g = sqrt(1.0 + qx * qx + qy * qy + qz * qz);
    const double vx = qx / g, vy = qy / g, vz = qz / g;
    // f_L = -(E + v x B) with that velocity
    const double fx = -(vy * bz - vz * by), fy = -(ey - vx * bz), fz = -(ez + vx * by);
    const double vE = vy * ey + vz * ez;
    const double sq = g * g * (fx * fx + fy * fy + fz * fz - vE * vE);
    // Eq. (f_r): f_R = -eps { f_L x B - (v.E) E + gamma^2 [f_L^2 - (v.E)^2] v }
    const double rx = -eps * ((fy * bz - fz * by) + sq * vx);
    const double ry = -eps * ((-fx * bz) - vE * ey + sq * vy);
    const double rz = -eps * ((fx * by) - vE * ez + sq * vz);
    // Eq. (pertfull): p^{n+1/2} = p_L^{n+1/2} + dt f_R
    p[0] = pLx + dt * rx;
    p[1] = pLy + dt * ry;
    p[2] = pLz + dt * rz;
}

__global__ void __launch_bounds__(ELEC_T) k_electron_leapfrog(const pic_electron_case* cases, int64_t n, double dt,
                                                               int64_t nsteps, int every, double eps, int flags,
                                                               double* out, int64_t nsamples) {
    const int64_t c = static_cast<int64_t>(blockIdx.x) * ELEC_T + threadIdx.x;
    if (c >= n) return;
    const pic_electron_case C = cases[c];
    const Wave w{C.wave, C.a0, C.tau};
    const bool rr = flags & 1;
    double x = C.x0, p[3] = {C.p0[0], C.p0[1], C.p0[2]};
    int64_t k = 0;
    for (int64_t s = 0; s < nsteps; ++s) {
        const double t = static_cast<double>(s) * dt;
        double ey, ez, dey, dez;
        wave_at(w, t - x, ey, ez, dey, dez);
        leapfrog_kick(p, ey, ez, dt, eps, rr);
        x += dt * p[0] / sqrt(1.0 + p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
        if ((s + 1) % every == 0 && k < nsamples) {
            double* o = out + (c * nsamples + k++) * 5;
            o[0] = static_cast<double>(s + 1) * dt;
            o[1] = x;
            o[2] = p[0];
            o[3] = p[1];
            o[4] = p[2];
        }
    }
}

}  // namespace

void launch_electron_scan(const pic_electron_case* cases, int64_t n, int integrator, int flags, double dt,
                          int64_t nsteps, int every, double eps, double* out, int64_t nsamples, cudaStream_t st) {
    const int64_t g = (n + ELEC_T - 1) / ELEC_T;
    if (integrator == PIC_INTEGRATOR_RK4)
        k_electron_rk4<<<static_cast<unsigned>(g), ELEC_T, 0, st>>>(cases, n, dt, nsteps, every, eps, flags, out,
                                                                    nsamples);
    else
        k_electron_leapfrog<<<static_cast<unsigned>(g), ELEC_T, 0, st>>>(cases, n, dt, nsteps, every, eps, flags,
                                                                         out, nsamples);
}

}  // namespace picrr

extern "C" pic_status pic_electron_scan(const pic_electron_case* cases, int64_t n, int integrator, int flags,
                                        double dt, int64_t nsteps, int every, double lambda_um, int device,
                                        double* out, int64_t nsamples) {
    using picrr::set_null_handle_error;
    if (n < 0 || n > (int64_t{1} << 31) || (n > 0 && (!cases || !out)))
        return set_null_handle_error("need 0 <= n <= 2^31 and non-NULL cases and out"), PIC_ERR_INVALID_ARG;
    if (integrator != PIC_INTEGRATOR_LEAPFROG && integrator != PIC_INTEGRATOR_RK4)
        return set_null_handle_error("unknown integrator"), PIC_ERR_INVALID_ARG;
    if ((flags & ~(PIC_ELECTRON_RR | PIC_ELECTRON_DERIV)) != 0 ||
        ((flags & PIC_ELECTRON_DERIV) && integrator != PIC_INTEGRATOR_RK4))
        return set_null_handle_error("bad flags (the derivative term is an RK4 option)"), PIC_ERR_INVALID_ARG;
    if (!(dt > 0.0) || nsteps < 0 || every < 1 || nsamples < 0 || nsamples > nsteps / every ||
        !(lambda_um > 0.0))
        return set_null_handle_error("need dt > 0, every >= 1, 0 <= nsamples <= nsteps/every, lambda_um > 0"),
               PIC_ERR_INVALID_ARG;
    for (int64_t c = 0; c < n; ++c)
        if (cases[c].wave < 0 || cases[c].wave > 2 || (cases[c].wave == 2 && !(cases[c].tau > 0.0)))
            return set_null_handle_error("bad wave (0, 1, or 2 with tau > 0)"), PIC_ERR_INVALID_ARG;
    if (n == 0) return PIC_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return set_null_handle_error("bad device"), PIC_ERR_INVALID_ARG;
    }
    const double eps = (4.0 / 3.0) * 3.14159265358979323846 * 2.8179403262e-9 / lambda_um;  // r_e in um (CODATA)
    cudaStream_t st = nullptr;
    pic_electron_case* dc = nullptr;
    double* dout = nullptr;
    const size_t out_bytes = static_cast<size_t>(n) * static_cast<size_t>(nsamples) * 5 * sizeof(double);
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocAsync(&dc, sizeof(pic_electron_case) * n, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&dout, out_bytes ? out_bytes : 16, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dc, cases, sizeof(pic_electron_case) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        picrr::launch_electron_scan(dc, n, integrator, flags, dt, nsteps, every, eps, dout, nsamples, st);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && out_bytes) e = cudaMemcpyAsync(out, dout, out_bytes, cudaMemcpyDeviceToHost, st);
    if (dc) cudaFreeAsync(dc, st);
    if (dout) cudaFreeAsync(dout, st);
    const cudaError_t e2 = st ? cudaStreamSynchronize(st) : cudaSuccess;
    if (st) cudaStreamDestroy(st);
    if (prev >= 0) cudaSetDevice(prev);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_null_handle_error(std::string("electron scan: ") + cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    return PIC_OK;
}
