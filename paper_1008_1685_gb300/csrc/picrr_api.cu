// Host side of the picrr C ABI: argument checks, device memory, the step
// loop (push kernel, Yee kernel, periodic sort), read-backs and counters.
// See include/picrr.h for the contract of every entry point.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <utility>
#include <vector>

#include "picrr.h"
#include "picrr_internal.cuh"

using namespace picrr;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kReUm = 2.8179403262e-9;    // classical electron radius, um (CODATA 2018)
constexpr double kMec2MeV = 0.51099895000;   // electron rest energy, MeV
constexpr double kMpMe = 1836.15267343;      // proton mass / electron mass
constexpr double kMuMe = 1822.888486209;     // atomic mass unit / electron mass
constexpr int kMaxDiagBlocks = 1024;

thread_local std::string g_create_error;  // failures of calls without a handle

struct HostSpecies {
    int64_t n = 0;
    bool loaded = false;
    DevSpecies buf[2] = {};
    int cur = 0;
    double w = 0.0, q = 0.0, m = 1.0;
};

struct EventPair {
    cudaEvent_t a, b;
    int kind;  // 0 push, 1 field, 2 sort
};

}  // namespace

namespace picrr {
void set_null_handle_error(const std::string& msg) { g_create_error = msg; }
}  // namespace picrr

struct pic_sim {
    pic_config cfg{};
    int Nx = 0, is = 8, sort_interval = 8, device = 0;
    double dx = 0, dt = 0, cfl = 0, eps = 0;
    cudaStream_t stream = nullptr, own_stream = nullptr;
    size_t bytes = 0, budget = 0;
    std::vector<std::pair<void*, size_t>> allocs;

    size_t glen = 0;
    float* F[2][5] = {};
    int fcur = 0;
    unsigned long long* Jacc[2][3] = {};
    float* Jf[3] = {};
    double* tally = nullptr;  // [4]
    int* status = nullptr;
    double* diag_partials = nullptr;
    double* diag_out = nullptr;  // [8]
    unsigned long long* bins = nullptr;
    int bins_cap = 0;

    HostSpecies sp[2];
    int max_units = 0;
    UnitTable units{};
    double* rad_part = nullptr;
    int32_t *cnt = nullptr, *offs = nullptr, *esc_cnt = nullptr, *esc_off = nullptr;
    int32_t *keycount[2] = {}, *keystart[2] = {}, *meta = nullptr;
    int32_t *blocksum[2] = {}, *blockstart[2] = {}, *tile_n[2] = {}, *tile_first[2] = {};

    int64_t step = 0;
    int since_sort = 0;
    bool prepared = false, laser_set = false, fields_set = false;
    LaserParams laser{};
    int fp_bits = 40;

    int64_t launches = 0, push_launches = 0, sorts = 0, timed_push = 0;
    bool timing = false;
    double push_ms = 0, field_ms = 0, sort_ms = 0;
    std::vector<EventPair> pending;
    std::vector<cudaEvent_t> ev_free;

    std::string err;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

pic_status fail(pic_sim* s, pic_status st, const std::string& msg) {
    if (s) s->err = msg;
    else g_create_error = msg;
    return st;
}

pic_status cuda_fail(pic_sim* s, cudaError_t e, const char* where) {
    return fail(s, PIC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define PIC_CK(s, call)                                         \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail((s), e_, #call); \
    } while (0)

// Allocate zeroed device memory charged to the handle's budget.  Appends to
// `fresh` so a failing call can release what it took.
pic_status dalloc(pic_sim* s, void** out, size_t bytes, std::vector<void*>* fresh) {
    *out = nullptr;
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~static_cast<size_t>(255);
    if (s->budget && s->bytes + bytes > s->budget)
        return fail(s, PIC_ERR_OOM, "device memory budget exceeded (" + std::to_string(s->bytes + bytes) +
                                        " > " + std::to_string(s->budget) + " bytes)");
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(s, PIC_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    e = cudaMemsetAsync(p, 0, bytes, s->stream);
    if (e != cudaSuccess) {
        cudaFree(p);
        return cuda_fail(s, e, "cudaMemsetAsync");
    }
    s->allocs.emplace_back(p, bytes);
    s->bytes += bytes;
    if (fresh) fresh->push_back(p);
    *out = p;
    return PIC_OK;
}

void dfree(pic_sim* s, void* p) {
    if (!p) return;
    for (size_t i = 0; i < s->allocs.size(); ++i) {
        if (s->allocs[i].first == p) {
            s->bytes -= s->allocs[i].second;
            s->allocs.erase(s->allocs.begin() + static_cast<long>(i));
            break;
        }
    }
    cudaFree(p);
}

void release(pic_sim* s, std::vector<void*>& fresh) {
    cudaStreamSynchronize(s->stream);
    for (void* p : fresh) dfree(s, p);
    fresh.clear();
}

template <class T>
pic_status dalloc_t(pic_sim* s, T** out, size_t count, std::vector<void*>* fresh) {
    void* p = nullptr;
    pic_status st = dalloc(s, &p, count * sizeof(T), fresh);
    *out = static_cast<T*>(p);
    return st;
}

pic_status alloc_species(pic_sim* s, HostSpecies& h, int64_t n, std::vector<void*>& fresh) {
    const size_t cap = static_cast<size_t>((n + 3) / 4 * 4 + 8);
    for (int b = 0; b < 2; ++b) {
        DevSpecies& d = h.buf[b];
        pic_status st;
        if ((st = dalloc_t(s, &d.cell, cap, &fresh)) != PIC_OK) return st;
        if ((st = dalloc_t(s, &d.off, cap, &fresh)) != PIC_OK) return st;
        if ((st = dalloc_t(s, &d.px, cap, &fresh)) != PIC_OK) return st;
        if ((st = dalloc_t(s, &d.py, cap, &fresh)) != PIC_OK) return st;
        if ((st = dalloc_t(s, &d.pz, cap, &fresh)) != PIC_OK) return st;
        if ((st = dalloc_t(s, &d.id, cap, &fresh)) != PIC_OK) return st;
    }
    h.n = n;
    h.cur = 0;
    return PIC_OK;
}

bool before_first_step(pic_sim* s) { return s->step == 0 && !s->prepared; }

cudaEvent_t take_event(pic_sim* s) {
    if (!s->ev_free.empty()) {
        cudaEvent_t e = s->ev_free.back();
        s->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Record an event pair around a launch sequence when timing is on.
struct Timed {
    pic_sim* s;
    EventPair ep{};
    bool on;
    Timed(pic_sim* sim, int kind) : s(sim), on(sim->timing) {
        if (on) {
            ep.a = take_event(s);
            ep.b = take_event(s);
            ep.kind = kind;
            cudaEventRecord(ep.a, s->stream);
        }
    }
    ~Timed() {
        if (on) {
            cudaEventRecord(ep.b, s->stream);
            s->pending.push_back(ep);
        }
    }
};

void collect_timing(pic_sim* s) {
    for (EventPair& ep : s->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ep.a, ep.b) == cudaSuccess) {
            if (ep.kind == 0) {
                s->push_ms += ms;
                s->timed_push++;
            } else if (ep.kind == 1) {
                s->field_ms += ms;
            } else {
                s->sort_ms += ms;
            }
        }
        s->ev_free.push_back(ep.a);
        s->ev_free.push_back(ep.b);
    }
    s->pending.clear();
}

SortParams sort_params(pic_sim* s) {
    SortParams S{};
    for (int k = 0; k < 2; ++k) {
        S.src[k] = s->sp[k].buf[s->sp[k].cur];
        S.dst[k] = s->sp[k].buf[1 - s->sp[k].cur];
        S.n[k] = s->sp[k].loaded ? s->sp[k].n : 0;
        S.keycount[k] = s->keycount[k];
        S.keystart[k] = s->keystart[k];
        S.blocksum[k] = s->blocksum[k];
        S.blockstart[k] = s->blockstart[k];
        S.tile_n[k] = s->tile_n[k];
        S.tile_first[k] = s->tile_first[k];
    }
    S.units = s->units;
    S.cnt = s->cnt;
    S.offs = s->offs;
    S.esc_cnt = s->esc_cnt;
    S.esc_off = s->esc_off;
    S.meta = s->meta;
    S.Nx = s->Nx;
    S.k = s->since_sort;
    S.max_units = s->max_units;
    return S;
}

// Allocate the unit table and sort scratch, fix the fixed-point scale and
// build the first unit table (particles are loaded in cell order).
pic_status prepare(pic_sim* s) {
    std::vector<void*> fresh;
    const int ntiles = (s->Nx + TILE - 1) / TILE;
    int64_t mu = 1;
    double bound = 0.0;
    for (int k = 0; k < 2; ++k) {
        if (!s->sp[k].loaded) continue;
        mu += (s->sp[k].n + UNIT_P - 1) / UNIT_P + ntiles + 1;
        bound += static_cast<double>(s->sp[k].n) * std::fabs(s->sp[k].q * s->sp[k].w) / s->cfl;
    }
    if (mu > (1 << 30)) return fail(s, PIC_ERR_INVALID_ARG, "too many work units");
    s->max_units = static_cast<int>(mu);
    // fixed point: every partial sum of the current is bounded by `bound`;
    // keep bound * 2^fp below 2^61.
    int fp = 40;
    if (bound > 0.0) fp = static_cast<int>(std::floor(61.0 - std::log2(bound)));
    s->fp_bits = std::max(8, std::min(52, fp));
    pic_status st;
    const size_t mu_z = static_cast<size_t>(mu);
    if ((st = dalloc_t(s, &s->units.species, mu_z, &fresh)) != PIC_OK) goto bad;
    if ((st = dalloc_t(s, &s->units.start, mu_z, &fresh)) != PIC_OK) goto bad;
    if ((st = dalloc_t(s, &s->units.end, mu_z, &fresh)) != PIC_OK) goto bad;
    if ((st = dalloc_t(s, &s->units.lo, mu_z, &fresh)) != PIC_OK) goto bad;
    if ((st = dalloc_t(s, &s->units.hi, mu_z, &fresh)) != PIC_OK) goto bad;
    if ((st = dalloc_t(s, &s->units.count, 4, &fresh)) != PIC_OK) goto bad;
    if ((st = dalloc_t(s, &s->rad_part, mu_z, &fresh)) != PIC_OK) goto bad;
    if ((st = dalloc_t(s, &s->cnt, mu_z * SSTR, &fresh)) != PIC_OK) goto bad;
    if ((st = dalloc_t(s, &s->offs, mu_z * SSTR, &fresh)) != PIC_OK) goto bad;
    if ((st = dalloc_t(s, &s->esc_cnt, mu_z, &fresh)) != PIC_OK) goto bad;
    if ((st = dalloc_t(s, &s->esc_off, mu_z, &fresh)) != PIC_OK) goto bad;
    for (int k = 0; k < 2; ++k) {
        if ((st = dalloc_t(s, &s->keycount[k], static_cast<size_t>(s->Nx) + 2, &fresh)) != PIC_OK) goto bad;
        if ((st = dalloc_t(s, &s->keystart[k], static_cast<size_t>(s->Nx) + 2, &fresh)) != PIC_OK) goto bad;
        const size_t nkb = static_cast<size_t>(s->Nx) / 256 + 2, ntl = static_cast<size_t>(s->Nx) / TILE + 3;
        if ((st = dalloc_t(s, &s->blocksum[k], nkb, &fresh)) != PIC_OK) goto bad;
        if ((st = dalloc_t(s, &s->blockstart[k], nkb, &fresh)) != PIC_OK) goto bad;
        if ((st = dalloc_t(s, &s->tile_n[k], ntl, &fresh)) != PIC_OK) goto bad;
        if ((st = dalloc_t(s, &s->tile_first[k], ntl, &fresh)) != PIC_OK) goto bad;
    }
    if ((st = dalloc_t(s, &s->meta, 8, &fresh)) != PIC_OK) goto bad;
    {
        // the loaded particles sit in buffer `cur` in cell order: build units from it
        SortParams S = sort_params(s);
        for (int k = 0; k < 2; ++k) S.dst[k] = s->sp[k].buf[s->sp[k].cur];
        int nl = 0;
        launch_build_units_from_sorted(S, s->stream, &nl);
        s->launches += nl;
        cudaError_t e = cudaStreamSynchronize(s->stream);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) {
            st = cuda_fail(s, e, "build units");
            goto bad;
        }
    }
    s->prepared = true;
    return PIC_OK;
bad:
    release(s, fresh);
    s->units = UnitTable{};
    s->rad_part = nullptr;
    s->cnt = s->offs = s->esc_cnt = s->esc_off = s->meta = nullptr;
    s->keycount[0] = s->keycount[1] = s->keystart[0] = s->keystart[1] = nullptr;
    for (int k = 0; k < 2; ++k) s->blocksum[k] = s->blockstart[k] = s->tile_n[k] = s->tile_first[k] = nullptr;
    return st;
}

PushParams push_params(pic_sim* s) {
    PushParams P{};
    for (int k = 0; k < 2; ++k) {
        const HostSpecies& h = s->sp[k];
        P.sp[k] = h.buf[h.cur];
        P.qm[k] = static_cast<float>(h.q / h.m);
        P.qw[k] = static_cast<float>(h.q * h.w);
        P.rad_w[k] = static_cast<float>(h.w * s->dx * h.m);
        P.rr[k] = (k == PIC_ELECTRON && s->cfg.rr_on) ? 1 : 0;
    }
    for (int c = 0; c < 5; ++c) P.F[c] = s->F[s->fcur][c];
    for (int c = 0; c < 3; ++c) P.J[c] = s->Jacc[s->step & 1][c];
    P.units = s->units;
    P.rad_part = s->rad_part;
    P.status = s->status;
    P.Nx = s->Nx;
    P.k = s->since_sort;
    P.cfl = static_cast<float>(s->cfl);
    P.dt = static_cast<float>(s->dt);
    P.eps = static_cast<float>(s->eps);
    for (int k = 0; k < 2; ++k) {
        // a warp record sums at most 16 particles of one lane (a thread holds at
        // most UNIT_P / PUSH_T + 4 particles of a unit) over 32 lanes, each value
        // bounded by |q w| max(1, 1/cfl): keep every lane below 2^26
        static_assert(UNIT_P / PUSH_T + 4 <= 16, "running record bound");
        const double vmax = std::fabs(s->sp[k].q * s->sp[k].w) * std::max(1.0, 1.0 / s->cfl);
        int ls = 40;
        if (vmax > 0.0) ls = static_cast<int>(std::floor(26.0 - std::log2(16.0 * vmax)));
        ls = std::min(ls, s->fp_bits);
        P.lscale[k] = std::ldexp(1.0f, ls);
        P.lshift[k] = s->fp_bits - ls;
    }
    return P;
}

// Incident field of the laser at retarded time t (double precision phase and
// envelope): Ey_inc = Bz_inc = ay, Ez_inc = -By_inc = az.  LP: ay = a0 g sin t;
// CP: a0/sqrt2 per component, ay = a g sin t, az = -a g cos t.
void incident(const LaserParams& L, double t, float* ay, float* az) {
    *ay = 0.f;
    *az = 0.f;
    if (!L.on || t < 0.0 || t > L.tau) return;
    double g;
    if (L.env == PIC_ENV_SIN2) {
        const double q = std::sin(kPi * t / L.tau);
        g = q * q;
    } else if (t < L.rise) {
        const double q = std::sin(0.5 * kPi * t / L.rise);
        g = q * q;
    } else if (t > L.tau - L.rise) {
        const double q = std::sin(0.5 * kPi * (L.tau - t) / L.rise);
        g = q * q;
    } else {
        g = 1.0;
    }
    if (L.pol == PIC_LP) {
        *ay = static_cast<float>(L.a0 * g * std::sin(t));
    } else {
        const double a = L.a0 / std::sqrt(2.0);
        *ay = static_cast<float>(a * g * std::sin(t));
        *az = static_cast<float>(-a * g * std::cos(t));
    }
}

FieldParams field_params(pic_sim* s) {
    FieldParams Q{};
    for (int c = 0; c < 5; ++c) {
        Q.Fo[c] = s->F[s->fcur][c];
        Q.Fn[c] = s->F[1 - s->fcur][c];
    }
    for (int c = 0; c < 3; ++c) {
        Q.Jacc[c] = s->Jacc[s->step & 1][c];
        Q.Jnext[c] = s->Jacc[(s->step + 1) & 1][c];
        Q.Jf[c] = s->Jf[c];
    }
    Q.tally = s->tally;
    Q.Nx = s->Nx;
    Q.is = s->is;
    Q.glen = static_cast<int>(s->glen);
    Q.n = s->step;
    Q.dt = s->dt;
    Q.dx = s->dx;
    Q.c = static_cast<float>(s->cfl);
    Q.hc = static_cast<float>(0.5 * s->cfl);
    Q.fdt = static_cast<float>(s->dt);
    Q.fp_inv = std::ldexp(1.0f, -s->fp_bits);
    const double tn = static_cast<double>(s->step) * s->dt;
    const double ts[3] = {tn, tn + 0.5 * s->dt + 0.5 * s->dx, tn + s->dt};
    for (int k = 0; k < 3; ++k) incident(s->laser, ts[k], &Q.inc[2 * k], &Q.inc[2 * k + 1]);
    return Q;
}

}  // namespace

// ============================================================================
extern "C" {

pic_status pic_create(const pic_config* cfg, pic_sim** out) {
    if (!out) return fail(nullptr, PIC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!cfg) return fail(nullptr, PIC_ERR_INVALID_ARG, "cfg is NULL");
    if (!(cfg->length_lambda > 0.0) || !(cfg->cells_per_lambda > 0.0))
        return fail(nullptr, PIC_ERR_INVALID_ARG, "length_lambda and cells_per_lambda must be > 0");
    if (!(cfg->cfl > 0.0 && cfg->cfl < 1.0)) return fail(nullptr, PIC_ERR_INVALID_ARG, "cfl must be in (0, 1)");
    if (!(cfg->lambda_um > 0.0)) return fail(nullptr, PIC_ERR_INVALID_ARG, "lambda_um must be > 0");
    if (cfg->sort_interval < 0 || cfg->sort_interval > KMAX)
        return fail(nullptr, PIC_ERR_INVALID_ARG, "sort_interval must be in [0, 32]");
    const double ncell = cfg->length_lambda * cfg->cells_per_lambda;
    if (!(ncell >= 16.0 && ncell <= 1.0e9)) return fail(nullptr, PIC_ERR_INVALID_ARG, "Nx must be in [16, 1e9]");
    const int Nx = static_cast<int>(std::llround(ncell));
    const int is = cfg->source_node ? cfg->source_node : 8;
    if (is < 2 || is > Nx - 4) return fail(nullptr, PIC_ERR_INVALID_ARG, "source_node must be in [2, Nx-4]");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(nullptr, PIC_ERR_CUDA, "no CUDA device");
    }
    if (cfg->device < 0 || cfg->device >= ndev) return fail(nullptr, PIC_ERR_INVALID_ARG, "device out of range");
    DeviceGuard g(cfg->device);

    pic_sim* s = new pic_sim();
    s->cfg = *cfg;
    s->device = cfg->device;
    s->Nx = Nx;
    s->is = is;
    s->sort_interval = cfg->sort_interval ? cfg->sort_interval : 8;
    s->dx = 2.0 * kPi / cfg->cells_per_lambda;
    s->cfl = cfg->cfl;
    s->dt = cfg->cfl * s->dx;
    s->eps = (4.0 / 3.0) * kPi * kReUm / cfg->lambda_um;
    s->budget = cfg->hbm_budget_bytes;
    if (cudaStreamCreateWithFlags(&s->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return fail(nullptr, PIC_ERR_CUDA, "cudaStreamCreate failed");
    }
    s->stream = s->own_stream;
    s->glen = (static_cast<size_t>(Nx) + 1 + 2 * PADF + 4 + 3) / 4 * 4;
    pic_status st = PIC_OK;
    for (int b = 0; b < 2 && st == PIC_OK; ++b)
        for (int c = 0; c < 5 && st == PIC_OK; ++c) st = dalloc_t(s, &s->F[b][c], s->glen, nullptr);
    for (int b = 0; b < 2 && st == PIC_OK; ++b)
        for (int c = 0; c < 3 && st == PIC_OK; ++c) st = dalloc_t(s, &s->Jacc[b][c], s->glen, nullptr);
    for (int c = 0; c < 3 && st == PIC_OK; ++c) st = dalloc_t(s, &s->Jf[c], s->glen, nullptr);
    if (st == PIC_OK) st = dalloc_t(s, &s->tally, 4, nullptr);
    if (st == PIC_OK) st = dalloc_t(s, &s->status, 4, nullptr);
    if (st == PIC_OK) st = dalloc_t(s, &s->diag_partials, kMaxDiagBlocks, nullptr);
    if (st == PIC_OK) st = dalloc_t(s, &s->diag_out, 8, nullptr);
    if (st == PIC_OK && cudaStreamSynchronize(s->stream) != cudaSuccess) st = PIC_ERR_CUDA;
    if (st != PIC_OK) {
        g_create_error = s->err;
        pic_destroy(s);
        return st;
    }
    *out = s;
    return PIC_OK;
}

pic_status pic_set_stream(pic_sim* s, void* stream) {
    if (!s) return PIC_ERR_INVALID_ARG;
    DeviceGuard g(s->device);
    cudaStreamSynchronize(s->stream);
    s->stream = stream ? static_cast<cudaStream_t>(stream) : s->own_stream;
    return PIC_OK;
}

pic_status pic_load_foil(pic_sim* s, double x0_lambda, double thickness_lambda, double ne_over_nc, int ion_Z,
                         double ion_A, int ppc) {
    if (!s) return PIC_ERR_INVALID_ARG;
    if (!before_first_step(s)) return fail(s, PIC_ERR_STATE, "load_foil after the first step");
    if (s->sp[0].loaded || s->sp[1].loaded) return fail(s, PIC_ERR_STATE, "particles already loaded");
    if (!(ne_over_nc > 0.0) || ion_Z < 1 || !(ion_A > 0.0) || ppc < 1)
        return fail(s, PIC_ERR_INVALID_ARG, "need ne > 0, Z >= 1, A > 0, ppc >= 1");
    const double cpl = s->cfg.cells_per_lambda;
    const long long c0 = std::llround(x0_lambda * cpl), nc = std::llround(thickness_lambda * cpl);
    if (!(std::isfinite(x0_lambda) && std::isfinite(thickness_lambda)) || c0 < 0 || nc < 1 || c0 + nc > s->Nx)
        return fail(s, PIC_ERR_INVALID_ARG, "foil must lie inside the box and span at least one cell");
    const long long n = nc * static_cast<long long>(ppc);
    if (n > 2147483647LL - 64) return fail(s, PIC_ERR_INVALID_ARG, "more than 2^31 particles per species");
    DeviceGuard g(s->device);
    std::vector<void*> fresh;
    pic_status st;
    for (int k = 0; k < 2; ++k)
        if ((st = alloc_species(s, s->sp[k], n, fresh)) != PIC_OK) {
            release(s, fresh);
            s->sp[0] = HostSpecies{};
            s->sp[1] = HostSpecies{};
            return st;
        }
    launch_foil(s->sp[0].buf[0], s->sp[1].buf[0], static_cast<int>(c0), static_cast<int>(nc), ppc, s->cfg.seed,
                s->stream);
    s->launches++;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        release(s, fresh);
        s->sp[0] = HostSpecies{};
        s->sp[1] = HostSpecies{};
        return cuda_fail(s, e, "foil loader");
    }
    HostSpecies& el = s->sp[0];
    HostSpecies& io = s->sp[1];
    el.q = -1.0;
    el.m = 1.0;
    el.w = ne_over_nc / ppc;
    io.q = ion_Z;
    io.m = (ion_Z == 1 && ion_A == 1.0) ? kMpMe : ion_A * kMuMe;
    io.w = ne_over_nc / (static_cast<double>(ion_Z) * ppc);
    el.loaded = io.loaded = true;
    return PIC_OK;
}

pic_status pic_load_particles(pic_sim* s, int species, int64_t n, const int32_t* cell, const double* off,
                              const double* px, const double* py, const double* pz, double weight, double charge,
                              double mass) {
    if (!s) return PIC_ERR_INVALID_ARG;
    if (species != PIC_ELECTRON && species != PIC_ION) return fail(s, PIC_ERR_INVALID_ARG, "bad species");
    if (!before_first_step(s)) return fail(s, PIC_ERR_STATE, "load_particles after the first step");
    if (s->sp[species].loaded) return fail(s, PIC_ERR_STATE, "species already loaded");
    if (n < 0 || n > 2147483647LL - 64) return fail(s, PIC_ERR_INVALID_ARG, "n must be in [0, 2^31 - 64]");
    if (n > 0 && (!cell || !off || !px || !py || !pz)) return fail(s, PIC_ERR_INVALID_ARG, "NULL array");
    if (!(mass > 0.0) || !std::isfinite(weight) || !std::isfinite(charge))
        return fail(s, PIC_ERR_INVALID_ARG, "mass must be > 0, weight and charge finite");
    std::vector<int32_t> hc(static_cast<size_t>(n)), hid(static_cast<size_t>(n));
    std::vector<float> ho(static_cast<size_t>(n)), hx(static_cast<size_t>(n)), hy(static_cast<size_t>(n)),
        hz(static_cast<size_t>(n));
    std::vector<int64_t> order(static_cast<size_t>(n));
    for (int64_t i = 0; i < n; ++i) {
        if (cell[i] < 0 || cell[i] >= s->Nx) return fail(s, PIC_ERR_INVALID_ARG, "cell out of [0, Nx)");
        const float o = static_cast<float>(off[i]);
        if (!(o >= 0.0f && o < 1.0f)) return fail(s, PIC_ERR_INVALID_ARG, "offset out of [0, 1) in float");
        if (!std::isfinite(px[i]) || !std::isfinite(py[i]) || !std::isfinite(pz[i]))
            return fail(s, PIC_ERR_INVALID_ARG, "non-finite momentum");
        order[static_cast<size_t>(i)] = i;
    }
    // the unit table needs particles in cell order: stable sort, ids keep the load order
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return cell[a] < cell[b]; });
    for (int64_t j = 0; j < n; ++j) {
        const int64_t i = order[static_cast<size_t>(j)];
        hc[j] = cell[i];
        ho[j] = static_cast<float>(off[i]);
        hx[j] = static_cast<float>(px[i]);
        hy[j] = static_cast<float>(py[i]);
        hz[j] = static_cast<float>(pz[i]);
        hid[j] = static_cast<int32_t>(i);
    }
    DeviceGuard g(s->device);
    std::vector<void*> fresh;
    HostSpecies h;
    pic_status st = alloc_species(s, h, n, fresh);
    if (st != PIC_OK) {
        release(s, fresh);
        return st;
    }
    const DevSpecies& d = h.buf[0];
    const size_t b4 = static_cast<size_t>(n) * 4;
    cudaError_t e = cudaSuccess;
    if (n > 0) {
        e = cudaMemcpyAsync(d.cell, hc.data(), b4, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d.off, ho.data(), b4, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d.px, hx.data(), b4, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d.py, hy.data(), b4, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d.pz, hz.data(), b4, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d.id, hid.data(), b4, cudaMemcpyHostToDevice, s->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        release(s, fresh);
        return cuda_fail(s, e, "upload particles");
    }
    h.w = weight;
    h.q = charge;
    h.m = mass;
    h.loaded = true;
    s->sp[species] = h;
    return PIC_OK;
}

pic_status pic_load_particles_f32(pic_sim* s, int species, int64_t n, const int32_t* cell, const float* off,
                                  const float* px, const float* py, const float* pz, double weight, double charge,
                                  double mass) {
    if (!s) return PIC_ERR_INVALID_ARG;
    if (species != PIC_ELECTRON && species != PIC_ION) return fail(s, PIC_ERR_INVALID_ARG, "bad species");
    if (!before_first_step(s)) return fail(s, PIC_ERR_STATE, "load_particles after the first step");
    if (s->sp[species].loaded) return fail(s, PIC_ERR_STATE, "species already loaded");
    if (n < 0 || n > 2147483647LL - 64) return fail(s, PIC_ERR_INVALID_ARG, "n must be in [0, 2^31 - 64]");
    if (n > 0 && (!cell || !off || !px || !py || !pz)) return fail(s, PIC_ERR_INVALID_ARG, "NULL array");
    if (!(mass > 0.0) || !std::isfinite(weight) || !std::isfinite(charge))
        return fail(s, PIC_ERR_INVALID_ARG, "mass must be > 0, weight and charge finite");
    bool sorted = true;
    for (int64_t i = 0; i < n; ++i) {
        if (cell[i] < 0 || cell[i] >= s->Nx) return fail(s, PIC_ERR_INVALID_ARG, "cell out of [0, Nx)");
        if (!(off[i] >= 0.0f && off[i] < 1.0f)) return fail(s, PIC_ERR_INVALID_ARG, "offset out of [0, 1)");
        if (!std::isfinite(px[i]) || !std::isfinite(py[i]) || !std::isfinite(pz[i]))
            return fail(s, PIC_ERR_INVALID_ARG, "non-finite momentum");
        if (i > 0 && cell[i] < cell[i - 1]) sorted = false;
    }
    if (!sorted) {
        std::vector<double> o(off, off + n), x(px, px + n), y(py, py + n), z(pz, pz + n);
        return pic_load_particles(s, species, n, cell, o.data(), x.data(), y.data(), z.data(), weight, charge,
                                  mass);
    }
    DeviceGuard g(s->device);
    std::vector<void*> fresh;
    HostSpecies h;
    pic_status st = alloc_species(s, h, n, fresh);
    if (st != PIC_OK) {
        release(s, fresh);
        return st;
    }
    const DevSpecies& d = h.buf[0];
    const size_t b4 = static_cast<size_t>(n) * 4;
    cudaError_t e = cudaSuccess;
    if (n > 0) {
        e = cudaMemcpyAsync(d.cell, cell, b4, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d.off, off, b4, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d.px, px, b4, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d.py, py, b4, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d.pz, pz, b4, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) {
            launch_iota(d.id, n, s->stream);
            s->launches++;
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        release(s, fresh);
        return cuda_fail(s, e, "upload particles");
    }
    h.w = weight;
    h.q = charge;
    h.m = mass;
    h.loaded = true;
    s->sp[species] = h;
    return PIC_OK;
}

pic_status pic_set_fields(pic_sim* s, const double* Ex, const double* Ey, const double* Ez, const double* By,
                          const double* Bz) {
    if (!s) return PIC_ERR_INVALID_ARG;
    if (!before_first_step(s)) return fail(s, PIC_ERR_STATE, "set_fields after the first step");
    if (s->fields_set) return fail(s, PIC_ERR_STATE, "fields already set");
    const double* src[5] = {Ex, Ey, Ez, By, Bz};
    std::vector<float> h(s->glen);
    DeviceGuard g(s->device);
    for (int c = 0; c < 5; ++c) {
        std::fill(h.begin(), h.end(), 0.0f);
        const int n = (c == 1 || c == 2) ? s->Nx + 1 : s->Nx;
        if (src[c])
            for (int i = 0; i < n; ++i) {
                if (!std::isfinite(src[c][i])) return fail(s, PIC_ERR_INVALID_ARG, "non-finite field value");
                h[PADF + i] = static_cast<float>(src[c][i]);
            }
        PIC_CK(s, cudaMemcpyAsync(s->F[s->fcur][c], h.data(), s->glen * 4, cudaMemcpyHostToDevice, s->stream));
        PIC_CK(s, cudaStreamSynchronize(s->stream));
    }
    s->fields_set = true;
    return PIC_OK;
}

pic_status pic_inject_laser(pic_sim* s, double a0, int polarization, int envelope, double duration_periods,
                            double rise_periods) {
    if (!s) return PIC_ERR_INVALID_ARG;
    if (!before_first_step(s)) return fail(s, PIC_ERR_STATE, "inject_laser after the first step");
    if (s->laser_set) return fail(s, PIC_ERR_STATE, "laser already set");
    if (!(a0 >= 0.0 && std::isfinite(a0))) return fail(s, PIC_ERR_INVALID_ARG, "a0 must be finite and >= 0");
    if (polarization != PIC_LP && polarization != PIC_CP) return fail(s, PIC_ERR_INVALID_ARG, "bad polarization");
    if (envelope != PIC_ENV_SIN2 && envelope != PIC_ENV_TRAPEZOID) return fail(s, PIC_ERR_INVALID_ARG, "bad envelope");
    if (!(duration_periods > 0.0 && std::isfinite(duration_periods)))
        return fail(s, PIC_ERR_INVALID_ARG, "duration must be > 0");
    if (envelope == PIC_ENV_TRAPEZOID && !(rise_periods > 0.0 && 2.0 * rise_periods <= duration_periods))
        return fail(s, PIC_ERR_INVALID_ARG, "trapezoid needs 0 < 2 rise <= duration");
    s->laser.on = 1;
    s->laser.pol = polarization;
    s->laser.env = envelope;
    s->laser.a0 = a0;
    s->laser.tau = duration_periods * 2.0 * kPi;
    s->laser.rise = rise_periods * 2.0 * kPi;
    s->laser_set = true;
    return PIC_OK;
}

// Add the per-unit radiated energy into the tally (before the units change).
static void rad_flush(pic_sim* s) {
    launch_rad_flush(s->rad_part, s->units.count, s->tally, s->stream);
    s->launches++;
}

static pic_status do_sort(pic_sim* s) {
    SortParams S = sort_params(s);
    int nl = 0;
    {
        Timed t(s, 2);
        rad_flush(s);
        launch_sort(S, s->max_units, s->stream, &nl);
    }
    s->launches += nl;
    for (int k = 0; k < 2; ++k) s->sp[k].cur ^= 1;
    s->sorts++;
    s->since_sort = 0;
    return PIC_OK;
}

pic_status pic_step_n(pic_sim* s, int64_t n, int64_t* steps_done) {
    if (steps_done) *steps_done = 0;
    if (!s) return PIC_ERR_INVALID_ARG;
    if (n < 0) return fail(s, PIC_ERR_INVALID_ARG, "n must be >= 0");
    DeviceGuard g(s->device);
    if (!s->prepared) {
        pic_status st = prepare(s);
        if (st != PIC_OK) return st;
    }
    const int fgrid = (s->Nx + 1 + FIELD_T - 1) / FIELD_T;
    for (int64_t it = 0; it < n; ++it) {
        {
            Timed t(s, 0);
            launch_push(push_params(s), s->max_units, s->stream);
        }
        {
            Timed t(s, 1);
            launch_field(field_params(s), fgrid, s->stream);
        }
        s->launches += 2;
        s->push_launches++;
        s->fcur ^= 1;
        s->step++;
        s->since_sort++;
        if (s->since_sort >= s->sort_interval) do_sort(s);
        if ((it & 255) == 255) {  // keep the host from running far ahead; surface launch errors early
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(s, e, "step launch");
        }
    }
    if (n > 0 && s->since_sort > 0) rad_flush(s);
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(s, e, "step");
    collect_timing(s);
    int hst[1] = {0}, meta[8] = {0};
    PIC_CK(s, cudaMemcpy(hst, s->status, sizeof(int), cudaMemcpyDeviceToHost));
    PIC_CK(s, cudaMemcpy(meta, s->meta, sizeof(meta), cudaMemcpyDeviceToHost));
    if (steps_done) *steps_done = n;
    if (hst[0] & ST_TIMEOUT) return fail(s, PIC_ERR_TIMEOUT, "a bounded device wait (TMA field window) gave up");
    if ((hst[0] | meta[4]) & ST_WINDOW) return fail(s, PIC_ERR_STATE, "a particle left its unit window");
    return PIC_OK;
}

pic_status pic_energy(pic_sim* s, double out[6]) {
    if (!s || !out) return s ? fail(s, PIC_ERR_INVALID_ARG, "out is NULL") : PIC_ERR_INVALID_ARG;
    DeviceGuard g(s->device);
    DiagParams D{};
    for (int c = 0; c < 5; ++c) D.F[c] = s->F[s->fcur][c];
    D.Nx = s->Nx;
    D.is = s->is;
    D.hc = static_cast<float>(0.5 * s->cfl);
    int nb = launch_field_energy(D, s->diag_partials, kMaxDiagBlocks, s->stream);
    launch_reduce_partials(s->diag_partials, nb, s->dx, s->diag_out + 0, s->stream);
    s->launches += 2;
    for (int k = 0; k < 2; ++k) {
        const HostSpecies& h = s->sp[k];
        if (!h.loaded || h.n == 0) {
            PIC_CK(s, cudaMemsetAsync(s->diag_out + 1 + k, 0, sizeof(double), s->stream));
            continue;
        }
        nb = launch_kinetic(h.buf[h.cur], h.n, s->diag_partials, kMaxDiagBlocks, s->stream);
        launch_reduce_partials(s->diag_partials, nb, h.w * s->dx * h.m, s->diag_out + 1 + k, s->stream);
        s->launches += 2;
    }
    double d[3], t[3];
    PIC_CK(s, cudaMemcpyAsync(d, s->diag_out, sizeof(d), cudaMemcpyDeviceToHost, s->stream));
    PIC_CK(s, cudaMemcpyAsync(t, s->tally, sizeof(t), cudaMemcpyDeviceToHost, s->stream));
    PIC_CK(s, cudaStreamSynchronize(s->stream));
    out[0] = d[0];
    out[1] = d[1];
    out[2] = d[2];
    out[3] = t[0];
    out[4] = t[1];
    out[5] = t[2];
    return PIC_OK;
}

pic_status pic_spectra(pic_sim* s, int species, int nbins, double e_min, double e_max, double* counts,
                       double* radiated) {
    if (!s) return PIC_ERR_INVALID_ARG;
    if (species != PIC_ELECTRON && species != PIC_ION) return fail(s, PIC_ERR_INVALID_ARG, "bad species");
    if (nbins < 1 || nbins > (1 << 24) || !counts || !(e_max > e_min) || !std::isfinite(e_min) ||
        !std::isfinite(e_max))
        return fail(s, PIC_ERR_INVALID_ARG, "need 1 <= nbins <= 2^24, e_max > e_min, counts != NULL");
    DeviceGuard g(s->device);
    const HostSpecies& h = s->sp[species];
    std::vector<unsigned long long> hb(static_cast<size_t>(nbins) + 2, 0ull);
    if (h.loaded && h.n > 0) {
        if (s->bins_cap < nbins + 2) {
            if (s->bins) dfree(s, s->bins);
            s->bins = nullptr;
            s->bins_cap = 0;
            pic_status st = dalloc_t(s, &s->bins, static_cast<size_t>(nbins) + 2, nullptr);
            if (st != PIC_OK) return st;
            s->bins_cap = nbins + 2;
        }
        PIC_CK(s, cudaMemsetAsync(s->bins, 0, sizeof(unsigned long long) * (nbins + 2), s->stream));
        launch_spectrum(h.buf[h.cur], h.n, h.m * kMec2MeV, nbins, e_min, e_max, s->bins, s->stream);
        s->launches++;
        PIC_CK(s, cudaMemcpyAsync(hb.data(), s->bins, sizeof(unsigned long long) * (nbins + 2),
                                  cudaMemcpyDeviceToHost, s->stream));
    }
    double tally0 = 0.0;
    PIC_CK(s, cudaMemcpyAsync(&tally0, s->tally, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    PIC_CK(s, cudaStreamSynchronize(s->stream));
    const double width = (e_max - e_min) / nbins;
    const double wdx = h.w * s->dx;
    for (int k = 0; k < nbins; ++k) counts[k] = static_cast<double>(hb[k]) * wdx / width;
    if (radiated) {
        // energy unit per area: m_e c^2 n_c (c/omega), n_c = eps0 m_e omega^2 / e^2 (SI)
        const double me = 9.1093837015e-31, c = 299792458.0, qe = 1.602176634e-19, eps0 = 8.8541878128e-12;
        const double omega = 2.0 * kPi * c / (s->cfg.lambda_um * 1e-6);
        const double nc = eps0 * me * omega * omega / (qe * qe);
        *radiated = tally0 * me * c * c * nc * c / omega;
    }
    return PIC_OK;
}

pic_status pic_read_particles(pic_sim* s, int species, int64_t cap, double* x, double* px, double* py, double* pz,
                              int32_t* flag, int64_t* nout) {
    if (!s) return PIC_ERR_INVALID_ARG;
    if (species != PIC_ELECTRON && species != PIC_ION) return fail(s, PIC_ERR_INVALID_ARG, "bad species");
    const HostSpecies& h = s->sp[species];
    const int64_t n = h.loaded ? h.n : 0;
    if (nout) *nout = n;
    if (cap <= 0 || n == 0) return PIC_OK;
    DeviceGuard g(s->device);
    std::vector<int32_t> c(n), id(n);
    std::vector<float> o(n), qx(n), qy(n), qz(n);
    const DevSpecies& d = h.buf[h.cur];
    const size_t b = static_cast<size_t>(n) * 4;
    PIC_CK(s, cudaMemcpyAsync(c.data(), d.cell, b, cudaMemcpyDeviceToHost, s->stream));
    PIC_CK(s, cudaMemcpyAsync(id.data(), d.id, b, cudaMemcpyDeviceToHost, s->stream));
    PIC_CK(s, cudaMemcpyAsync(o.data(), d.off, b, cudaMemcpyDeviceToHost, s->stream));
    PIC_CK(s, cudaMemcpyAsync(qx.data(), d.px, b, cudaMemcpyDeviceToHost, s->stream));
    PIC_CK(s, cudaMemcpyAsync(qy.data(), d.py, b, cudaMemcpyDeviceToHost, s->stream));
    PIC_CK(s, cudaMemcpyAsync(qz.data(), d.pz, b, cudaMemcpyDeviceToHost, s->stream));
    PIC_CK(s, cudaStreamSynchronize(s->stream));
    for (int64_t i = 0; i < n; ++i) {
        const int64_t j = id[i];
        if (j < 0 || j >= n) return fail(s, PIC_ERR_STATE, "corrupt particle id");
        if (j >= cap) continue;
        int fl = 0;
        double xi;
        if (c[i] == -1) {
            xi = 0.0;
            fl = -1;
        } else if (c[i] == -2) {
            xi = s->Nx;
            fl = 1;
        } else {
            xi = static_cast<double>(c[i]) + o[i];
        }
        if (x) x[j] = xi * s->dx;
        if (px) px[j] = qx[i];
        if (py) py[j] = qy[i];
        if (pz) pz[j] = qz[i];
        if (flag) flag[j] = fl;
    }
    return PIC_OK;
}

pic_status pic_read_fields(pic_sim* s, int comp, int64_t cap, double* out, int64_t* nout) {
    if (!s) return PIC_ERR_INVALID_ARG;
    if (comp < PIC_EX || comp > PIC_JZ) return fail(s, PIC_ERR_INVALID_ARG, "bad component");
    const bool node = comp == PIC_EY || comp == PIC_EZ || comp == PIC_JY || comp == PIC_JZ;
    const int64_t n = node ? s->Nx + 1 : s->Nx;
    if (nout) *nout = n;
    if (!out || cap < n) return fail(s, PIC_ERR_INVALID_ARG, "output too small");
    DeviceGuard g(s->device);
    const float* src = comp <= PIC_BZ ? s->F[s->fcur][comp] : s->Jf[comp - PIC_JX];
    std::vector<float> h(static_cast<size_t>(n));
    PIC_CK(s, cudaMemcpyAsync(h.data(), src + PADF, sizeof(float) * n, cudaMemcpyDeviceToHost, s->stream));
    PIC_CK(s, cudaStreamSynchronize(s->stream));
    for (int64_t i = 0; i < n; ++i) out[i] = h[static_cast<size_t>(i)];
    return PIC_OK;
}

pic_status pic_stats(pic_sim* s, pic_stats_t* out) {
    if (!s || !out) return PIC_ERR_INVALID_ARG;
    DeviceGuard g(s->device);
    std::memset(out, 0, sizeof(*out));
    out->steps = s->step;
    out->kernel_launches = s->launches;
    out->push_launches = s->push_launches;
    out->sort_count = s->sorts;
    out->push_ms = s->push_ms;
    out->field_ms = s->field_ms;
    out->sort_ms = s->sort_ms;
    out->timed_push_launches = s->timed_push;
    out->device_bytes = static_cast<int64_t>(s->bytes);
    out->fp_bits = s->fp_bits;
    if (s->prepared) {
        int32_t cnt[4] = {0}, meta[8] = {0};
        PIC_CK(s, cudaMemcpyAsync(cnt, s->units.count, sizeof(cnt), cudaMemcpyDeviceToHost, s->stream));
        PIC_CK(s, cudaMemcpyAsync(meta, s->meta, sizeof(meta), cudaMemcpyDeviceToHost, s->stream));
        PIC_CK(s, cudaStreamSynchronize(s->stream));
        out->n_units = cnt[0];
        out->active_particles = static_cast<int64_t>(meta[0]) + meta[1];
    } else {
        out->active_particles = (s->sp[0].loaded ? s->sp[0].n : 0) + (s->sp[1].loaded ? s->sp[1].n : 0);
    }
    return PIC_OK;
}

pic_status pic_set_timing(pic_sim* s, int on) {
    if (!s) return PIC_ERR_INVALID_ARG;
    DeviceGuard g(s->device);
    cudaStreamSynchronize(s->stream);
    collect_timing(s);
    s->timing = on != 0;
    if (s->timing) {
        s->push_ms = s->field_ms = s->sort_ms = 0.0;
        s->timed_push = 0;
    }
    return PIC_OK;
}

const char* pic_last_error(const pic_sim* s) { return s ? s->err.c_str() : g_create_error.c_str(); }

pic_status pic_destroy(pic_sim* s) {
    if (!s) return PIC_OK;
    {
        DeviceGuard g(s->device);
        if (s->stream) cudaStreamSynchronize(s->stream);
        for (EventPair& ep : s->pending) {
            cudaEventDestroy(ep.a);
            cudaEventDestroy(ep.b);
        }
        for (cudaEvent_t e : s->ev_free) cudaEventDestroy(e);
        for (auto& a : s->allocs) cudaFree(a.first);
        s->allocs.clear();
        if (s->own_stream) cudaStreamDestroy(s->own_stream);
    }
    delete s;
    return PIC_OK;
}

}  // extern "C"
