// Host side of the picrr C ABI.
//
// Everything runs on a Batch: R independent runs (each its own grid, foil,
// laser, particle arrays) stepped together, one launch per kernel per step
// for all active runs.  A pic_sim handle is a batch of one run; a pic_batch
// handle exposes the batch itself.  The host side does argument checks,
// device memory (stream-ordered allocation charged to a budget), the device
// run table, the laser source values of each step (double precision), the
// step loop (push kernel, Yee kernel, periodic sort), read-backs and
// counters.  See include/picrr.h for the contract of every entry point.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "picrr.h"
#include "picrr_internal.cuh"

namespace picrr {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kReUm = 2.8179403262e-9;   // classical electron radius, um (CODATA 2018)
constexpr double kMec2MeV = 0.51099895000;  // electron rest energy, MeV
constexpr double kMpMe = 1836.15267343;     // proton mass / electron mass
constexpr double kMuMe = 1822.888486209;    // atomic mass unit / electron mass
constexpr double kLambdaCUm = 3.8615926796e-7;  // reduced Compton wavelength hbar/(m_e c), um (CODATA 2018)
constexpr int kMaxDiagBlocks = 1024;
constexpr int kIncRing = 16;                // slots of the laser-source upload ring (one chunk of steps each)

thread_local std::string g_null_error;  // failures of calls without a handle

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

struct HostSpecies {
    int64_t n = 0;
    bool loaded = false;
    double w = 0.0, q = 0.0, m = 1.0;
};

struct EventPair {
    cudaEvent_t a, b;
    int kind;  // 0 push, 1 field, 2 sort
};

}  // namespace

void set_null_handle_error(const std::string& msg) { g_null_error = msg; }

// Incident field of the laser at retarded time t (double precision phase and
// envelope): Ey_inc = Bz_inc = ay, Ez_inc = -By_inc = az.  LP: ay = a0 g sin t;
// CP: a0/sqrt2 per component, ay = a g sin t, az = -a g cos t.
static void incident(const LaserParams& L, double t, float* ay, float* az) {
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

// One run of a batch, host side.
struct RunHost {
    bool used = false;      // slot holds a run
    bool active = false;    // stepped by the batch
    bool started = false;   // took part in at least one step (setup frozen)
    bool finished = false;  // reached its step count
    double length_lambda = 0.0;
    int Nx = 0, is = 8, rr = 1;
    uint64_t seed = 1;
    HostSpecies sp[2];
    LaserParams laser{};
    bool laser_set = false, fields_set = false;
    int64_t admit_step = 0;    // batch step of its first step
    int64_t t_offset = 0;      // steps the run had made before it was restored from a checkpoint
    int64_t steps_target = 0;  // 0: unlimited
    int64_t steps_done = 0;
    int pbuf = 0, fbuf = 0;    // particle / field buffer of a finished run
    int fp_bits = 40;
    size_t glen = 0;
    std::vector<std::pair<void*, size_t>> mem;  // device allocations of this run
    RunDev dev{};                               // mirror of the device table entry
};

struct Batch {
    pic_config cfg{};
    int device = 0, sort_interval = 8, max_runs = 1;
    int unit_p = UNIT_P;  // particles per work unit at most (a run-time shape)
    int slot_w = 2;       // particles per thread and round of the push kernel (2 or 4; the tuner picks)
    double dx = 0, dt = 0, cfl = 0, eps = 0;
    cudaStream_t stream = nullptr, own_stream = nullptr;
    size_t bytes = 0, budget = 0;
    std::vector<std::pair<void*, size_t>> mem;  // batch-level allocations

    std::vector<RunHost> runs;
    RunDev* d_runs = nullptr;
    RunDev* h_runs = nullptr;  // pinned staging of the run table
    int32_t* d_blk_run = nullptr;
    int32_t* d_blk_i0 = nullptr;
    int nblk = 0, blk_cap = 0;
    float* d_inc = nullptr;  // [KMAX][max_runs * 6]
    float* h_inc = nullptr;  // pinned ring [kIncRing][KMAX][max_runs * 6]
    cudaEvent_t inc_ev[kIncRing] = {};
    int inc_slot = 0;

    // CUDA graphs of one sort interval of steps (its pushes, Yee updates and
    // the sort that ends it), by [step parity at the chunk start][current
    // particle buffer].  The kernels read the run table at run time, so a
    // graph stays valid while launch shapes and table pointers do (epoch).
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph[2][2] = {};
    uint64_t graph_epoch[2][2] = {};
    uint64_t epoch = 1;
    bool graphs_on = true;
    int64_t graph_launches = 0;
    // With timing on, the graphs also hold event-record nodes around every
    // push, Yee update and the sort: the event pairs of each graph, whether it
    // was captured with them, and whether a launch of it has not been read yet
    // (it is read before the same graph is launched again).
    std::vector<EventPair> graph_ev[2][2];
    bool graph_timed[2][2] = {};
    bool graph_unread[2][2] = {};

    UnitTable units{};
    int max_units = 0;
    double* rad_part = nullptr;
    int32_t *cnt = nullptr, *offs = nullptr, *rs_units = nullptr;
    int* d_status = nullptr;
    double* diag_partials = nullptr;
    double* diag_out = nullptr;
    unsigned long long* snap_out = nullptr;  // [4]: max d bits, max chi bits, flagged count
    unsigned long long* bins = nullptr;
    int bins_cap = 0;

    int64_t gstep = 0;
    int since_sort = 0;
    int cur = 0;
    bool table_dirty = true, layout_dirty = true;

    int64_t launches = 0, push_launches = 0, sorts = 0, timed_push = 0;
    bool timing = false;
    double push_ms = 0, field_ms = 0, sort_ms = 0;
    std::vector<EventPair> pending;
    std::vector<cudaEvent_t> ev_free;

    std::string err;
};

namespace {

pic_status fail(Batch* b, pic_status st, const std::string& msg) {
    if (b) b->err = msg;
    else g_null_error = msg;
    return st;
}

pic_status cuda_fail(Batch* b, cudaError_t e, const char* where) {
    cudaGetLastError();
    return fail(b, PIC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define PIC_CK(b, call)                                          \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail((b), e_, #call); \
    } while (0)

// Stream-ordered, zeroed device allocation charged to the batch's budget.
pic_status dalloc(Batch* b, std::vector<std::pair<void*, size_t>>& owner, void** out, size_t bytes) {
    *out = nullptr;
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~static_cast<size_t>(255);
    if (b->budget && b->bytes + bytes > b->budget)
        return fail(b, PIC_ERR_OOM, "device memory budget exceeded (" + std::to_string(b->bytes + bytes) + " > " +
                                        std::to_string(b->budget) + " bytes)");
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes, b->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(b, PIC_ERR_OOM, std::string("device allocation: ") + cudaGetErrorString(e));
    }
    e = cudaMemsetAsync(p, 0, bytes, b->stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(p, b->stream);
        return cuda_fail(b, e, "cudaMemsetAsync");
    }
    owner.emplace_back(p, bytes);
    b->bytes += bytes;
    *out = p;
    return PIC_OK;
}

template <class T>
pic_status dalloc_t(Batch* b, std::vector<std::pair<void*, size_t>>& owner, T** out, size_t count) {
    void* p = nullptr;
    pic_status st = dalloc(b, owner, &p, count * sizeof(T));
    *out = static_cast<T*>(p);
    return st;
}

void free_all(Batch* b, std::vector<std::pair<void*, size_t>>& owner) {
    for (auto& a : owner) {
        cudaFreeAsync(a.first, b->stream);
        b->bytes -= a.second;
    }
    owner.clear();
}

// Free allocations made after index `mark` of `owner` (undo of a failed call).
void free_from(Batch* b, std::vector<std::pair<void*, size_t>>& owner, size_t mark) {
    while (owner.size() > mark) {
        cudaFreeAsync(owner.back().first, b->stream);
        b->bytes -= owner.back().second;
        owner.pop_back();
    }
}

// Free one batch-level allocation.
void free_one(Batch* b, void* p) {
    if (!p) return;
    for (size_t i = 0; i < b->mem.size(); ++i)
        if (b->mem[i].first == p) {
            cudaFreeAsync(p, b->stream);
            b->bytes -= b->mem[i].second;
            b->mem.erase(b->mem.begin() + static_cast<long>(i));
            return;
        }
}

cudaEvent_t take_event(Batch* b) {
    if (!b->ev_free.empty()) {
        cudaEvent_t e = b->ev_free.back();
        b->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct Timed {
    Batch* b;
    EventPair ep{};
    bool on;
    Timed(Batch* bb, int kind) : b(bb), on(bb->timing) {
        if (on) {
            ep.a = take_event(b);
            ep.b = take_event(b);
            ep.kind = kind;
            cudaEventRecord(ep.a, b->stream);
        }
    }
    ~Timed() {
        if (on) {
            cudaEventRecord(ep.b, b->stream);
            b->pending.push_back(ep);
        }
    }
};

void add_timing(Batch* b, const EventPair& ep) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ep.a, ep.b) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (ep.kind == 0) {
        b->push_ms += ms;
        b->timed_push++;
    } else if (ep.kind == 1) {
        b->field_ms += ms;
    } else {
        b->sort_ms += ms;
    }
}

void collect_timing(Batch* b) {
    for (EventPair& ep : b->pending) {
        add_timing(b, ep);
        b->ev_free.push_back(ep.a);
        b->ev_free.push_back(ep.b);
    }
    b->pending.clear();
}

// Times of the last launch of chunk graph [par0][cur] (waits for its last event).
void read_graph_timing(Batch* b, int par0, int cur) {
    if (!b->graph_unread[par0][cur]) return;
    b->graph_unread[par0][cur] = false;
    const std::vector<EventPair>& ev = b->graph_ev[par0][cur];
    if (ev.empty() || cudaEventSynchronize(ev.back().b) != cudaSuccess) return;
    for (const EventPair& ep : ev) add_timing(b, ep);
}

void read_all_graph_timing(Batch* b) {
    for (int p = 0; p < 2; ++p)
        for (int c = 0; c < 2; ++c) read_graph_timing(b, p, c);
}

// Drop graph [par0][cur] and give its events back (after reading them).
void drop_graph(Batch* b, int par0, int cur) {
    read_graph_timing(b, par0, cur);
    if (b->graph[par0][cur]) cudaGraphExecDestroy(b->graph[par0][cur]);
    b->graph[par0][cur] = nullptr;
    for (EventPair& ep : b->graph_ev[par0][cur]) {
        b->ev_free.push_back(ep.a);
        b->ev_free.push_back(ep.b);
    }
    b->graph_ev[par0][cur].clear();
    b->graph_timed[par0][cur] = false;
}

// ---------------------------------------------------------------------------
// batch life cycle
// ---------------------------------------------------------------------------

pic_status validate_common(const pic_config* cfg) {
    if (!cfg) return fail(nullptr, PIC_ERR_INVALID_ARG, "cfg is NULL");
    if (!(cfg->cells_per_lambda > 0.0) || !std::isfinite(cfg->cells_per_lambda))
        return fail(nullptr, PIC_ERR_INVALID_ARG, "cells_per_lambda must be > 0");
    if (!(cfg->cfl > 0.0 && cfg->cfl < 1.0)) return fail(nullptr, PIC_ERR_INVALID_ARG, "cfl must be in (0, 1)");
    if (!(cfg->lambda_um > 0.0)) return fail(nullptr, PIC_ERR_INVALID_ARG, "lambda_um must be > 0");
    if (cfg->sort_interval < 0 || cfg->sort_interval > KMAX)
        return fail(nullptr, PIC_ERR_INVALID_ARG, "sort_interval must be in [0, 96]");
    return PIC_OK;
}

void batch_destroy(Batch* b);

pic_status batch_create(const pic_config* cfg, int max_runs, Batch** out) {
    *out = nullptr;
    pic_status st = validate_common(cfg);
    if (st != PIC_OK) return st;
    if (max_runs < 1 || max_runs > 8192) return fail(nullptr, PIC_ERR_INVALID_ARG, "max_runs must be in [1, 8192]");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(nullptr, PIC_ERR_CUDA, "no CUDA device");
    }
    if (cfg->device < 0 || cfg->device >= ndev) return fail(nullptr, PIC_ERR_INVALID_ARG, "device out of range");
    DeviceGuard g(cfg->device);
    Batch* b = new Batch();
    b->cfg = *cfg;
    b->device = cfg->device;
    b->max_runs = max_runs;
    b->sort_interval = cfg->sort_interval ? cfg->sort_interval : 8;
    b->dx = 2.0 * kPi / cfg->cells_per_lambda;
    b->cfl = cfg->cfl;
    b->dt = cfg->cfl * b->dx;
    b->eps = (4.0 / 3.0) * kPi * kReUm / cfg->lambda_um;
    b->budget = cfg->hbm_budget_bytes;
    b->runs.resize(static_cast<size_t>(max_runs));
    if (cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return fail(nullptr, PIC_ERR_CUDA, "cudaStreamCreate failed");
    }
    b->stream = b->own_stream;
    if ((st = dalloc_t(b, b->mem, &b->d_runs, static_cast<size_t>(max_runs))) != PIC_OK ||
        (st = dalloc_t(b, b->mem, &b->d_inc, static_cast<size_t>(max_runs) * 6 * KMAX)) != PIC_OK ||
        (st = dalloc_t(b, b->mem, &b->d_status, 4)) != PIC_OK ||
        (st = dalloc_t(b, b->mem, &b->diag_partials, kMaxDiagBlocks)) != PIC_OK ||
        (st = dalloc_t(b, b->mem, &b->diag_out, 8)) != PIC_OK ||
        (st = dalloc_t(b, b->mem, &b->snap_out, 4)) != PIC_OK ||
        (st = dalloc_t(b, b->mem, &b->rs_units, static_cast<size_t>(4) * max_runs)) != PIC_OK) {
        g_null_error = b->err;
        batch_destroy(b);
        return st;
    }
    if (cudaMallocHost(&b->h_runs, sizeof(RunDev) * max_runs) != cudaSuccess ||
        cudaMallocHost(&b->h_inc, sizeof(float) * 6 * max_runs * KMAX * kIncRing) != cudaSuccess) {
        cudaGetLastError();
        batch_destroy(b);
        return fail(nullptr, PIC_ERR_OOM, "pinned host allocation failed");
    }
    std::memset(b->h_runs, 0, sizeof(RunDev) * max_runs);
    for (int i = 0; i < kIncRing; ++i) cudaEventCreateWithFlags(&b->inc_ev[i], cudaEventDisableTiming);
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        batch_destroy(b);
        return fail(nullptr, PIC_ERR_CUDA, "cudaStreamCreate failed");
    }
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaError_t e = cudaGetLastError();
        batch_destroy(b);
        return cuda_fail(nullptr, e, "create");
    }
    *out = b;
    return PIC_OK;
}

void batch_destroy(Batch* b) {
    if (!b) return;
    DeviceGuard g(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (EventPair& ep : b->pending) {
        cudaEventDestroy(ep.a);
        cudaEventDestroy(ep.b);
    }
    for (cudaEvent_t e : b->ev_free) cudaEventDestroy(e);
    for (auto& r : b->runs) free_all(b, r.mem);
    free_all(b, b->mem);
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (int i = 0; i < kIncRing; ++i)
        if (b->inc_ev[i]) cudaEventDestroy(b->inc_ev[i]);
    if (b->h_runs) cudaFreeHost(b->h_runs);
    if (b->h_inc) cudaFreeHost(b->h_inc);
    for (int p = 0; p < 2; ++p)
        for (int c = 0; c < 2; ++c) {
            if (b->graph[p][c]) cudaGraphExecDestroy(b->graph[p][c]);
            for (EventPair& ep : b->graph_ev[p][c]) {
                cudaEventDestroy(ep.a);
                cudaEventDestroy(ep.b);
            }
        }
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->own_stream) cudaStreamDestroy(b->own_stream);
    delete b;
}

// New run slot with its grid arrays allocated (no particles yet).
pic_status run_open(Batch* b, double length_lambda, int source_node, int rr_on, uint64_t seed, int* out_id) {
    const double ncell = length_lambda * b->cfg.cells_per_lambda;
    if (!(length_lambda > 0.0) || !(ncell >= 16.0 && ncell <= 1.0e9))
        return fail(b, PIC_ERR_INVALID_ARG, "length_lambda * cells_per_lambda must be in [16, 1e9]");
    const int Nx = static_cast<int>(std::llround(ncell));
    const int is = source_node ? source_node : 8;
    if (is < 2 || is > Nx - 4) return fail(b, PIC_ERR_INVALID_ARG, "source_node must be in [2, Nx-4]");
    int id = -1;
    for (int i = 0; i < b->max_runs; ++i)
        if (!b->runs[i].used) {
            id = i;
            break;
        }
    if (id < 0) return fail(b, PIC_ERR_STATE, "no free run slot (max_runs reached)");
    RunHost& r = b->runs[id];
    r = RunHost();
    r.length_lambda = length_lambda;
    r.Nx = Nx;
    r.is = is;
    r.rr = rr_on ? 1 : 0;
    r.seed = seed;
    r.glen = (static_cast<size_t>(Nx) + 1 + 2 * PADF + 4 + 3) / 4 * 4;
    RunDev& d = r.dev;
    d.Nx = Nx;
    d.is = is;
    d.glen = static_cast<int>(r.glen);
    d.rr = r.rr;
    pic_status st = PIC_OK;
    for (int x = 0; x < 2 && st == PIC_OK; ++x)
        for (int c = 0; c < 5 && st == PIC_OK; ++c) st = dalloc_t(b, r.mem, &d.F[x][c], r.glen);
    for (int x = 0; x < 2 && st == PIC_OK; ++x)
        for (int c = 0; c < 3 && st == PIC_OK; ++c) st = dalloc_t(b, r.mem, &d.J[x][c], r.glen);
    if (st == PIC_OK) st = dalloc_t(b, r.mem, &d.tally, 4);
    const size_t nk = static_cast<size_t>(Nx) + 2, nkb = static_cast<size_t>(Nx) / KEY_T + 2,
                 ntl = static_cast<size_t>(Nx) / TILE + 3;
    for (int s = 0; s < 2 && st == PIC_OK; ++s) {
        if (st == PIC_OK) st = dalloc_t(b, r.mem, &d.keycount[s], nk);
        if (st == PIC_OK) st = dalloc_t(b, r.mem, &d.keystart[s], nk);
        if (st == PIC_OK) st = dalloc_t(b, r.mem, &d.blocksum[s], nkb);
        if (st == PIC_OK) st = dalloc_t(b, r.mem, &d.blockstart[s], nkb);
        if (st == PIC_OK) st = dalloc_t(b, r.mem, &d.tile_n[s], ntl);
        if (st == PIC_OK) st = dalloc_t(b, r.mem, &d.tile_first[s], ntl);
    }
    if (st != PIC_OK) {
        free_all(b, r.mem);
        r = RunHost();
        return st;
    }
    r.used = true;
    *out_id = id;
    return PIC_OK;
}

size_t rounded(size_t bytes) { return ((bytes ? bytes : 16) + 255) & ~static_cast<size_t>(255); }

// Device bytes a run of length_lambda with n particles per species takes in a
// batch: its grid, sort scratch and particle buffers as run_open and
// alloc_species allocate them, plus its share of the batch's unit table and
// Yee block table with the unit table's growth factor (1.5).
size_t run_footprint_cpl(double cells_per_lambda, double length_lambda, int64_t n) {
    const int64_t Nx = std::llround(length_lambda * cells_per_lambda);
    const size_t glen = (static_cast<size_t>(Nx) + 1 + 2 * PADF + 4 + 3) / 4 * 4;
    size_t t = 10 * rounded(glen * 4) + 6 * rounded(glen * 8) + 3 * rounded(glen * 4) + rounded(32);
    const size_t nk = static_cast<size_t>(Nx) + 2, nkb = static_cast<size_t>(Nx) / KEY_T + 2,
                 ntl = static_cast<size_t>(Nx) / TILE + 3;
    t += 2 * (2 * rounded(nk * 4) + 2 * rounded(nkb * 4) + 2 * rounded(ntl * 4));
    const size_t cap = static_cast<size_t>((n + 3) / 4 * 4 + 8);
    t += 2 * 2 * 6 * rounded(cap * 4);
    const int64_t ntiles = (Nx + TILE - 1) / TILE;
    const size_t units = static_cast<size_t>(2 * ((n + UNIT_P_MIN - 1) / UNIT_P_MIN + ntiles + 1));
    t += units * (6 * 4 + 8 + 2 * SSTR * 4) * 3 / 2;
    t += static_cast<size_t>(Nx / FIELD_NODES + 1) * 8 * 3 / 2;
    return t;
}

size_t run_footprint(const Batch* b, double length_lambda, int64_t n) {
    return run_footprint_cpl(b->cfg.cells_per_lambda, length_lambda, n);
}

void run_release(Batch* b, int id) {
    RunHost& r = b->runs[id];
    if (!r.used) return;
    if (r.active) b->layout_dirty = true;
    b->table_dirty = true;
    free_all(b, r.mem);
    r = RunHost();
}

pic_status alloc_species(Batch* b, RunHost& r, int s, int64_t n) {
    const size_t cap = static_cast<size_t>((n + 3) / 4 * 4 + 8);
    pic_status st = PIC_OK;
    for (int x = 0; x < 2 && st == PIC_OK; ++x) {
        DevSpecies& d = r.dev.sp[s][x];
        if (st == PIC_OK) st = dalloc_t(b, r.mem, &d.cell, cap);
        if (st == PIC_OK) st = dalloc_t(b, r.mem, &d.off, cap);
        if (st == PIC_OK) st = dalloc_t(b, r.mem, &d.px, cap);
        if (st == PIC_OK) st = dalloc_t(b, r.mem, &d.py, cap);
        if (st == PIC_OK) st = dalloc_t(b, r.mem, &d.pz, cap);
        if (st == PIC_OK) st = dalloc_t(b, r.mem, &d.id, cap);
    }
    if (st == PIC_OK) {
        r.sp[s].n = n;
        r.dev.n[s] = static_cast<int32_t>(n);
    }
    return st;
}

void clear_species(RunHost& r, int s) {
    r.sp[s] = HostSpecies();
    r.dev.n[s] = 0;
    for (int x = 0; x < 2; ++x) r.dev.sp[s][x] = DevSpecies{};
}

pic_status run_load_foil(Batch* b, int id, double x0_lambda, double thickness_lambda, double ne_over_nc, int ion_Z,
                         double ion_A, int ppc) {
    RunHost& r = b->runs[id];
    if (r.started) return fail(b, PIC_ERR_STATE, "load_foil after the first step");
    if (r.sp[0].loaded || r.sp[1].loaded) return fail(b, PIC_ERR_STATE, "particles already loaded");
    if (!(ne_over_nc > 0.0) || !std::isfinite(ne_over_nc) || ion_Z < 1 || !(ion_A > 0.0) || ppc < 1)
        return fail(b, PIC_ERR_INVALID_ARG, "need ne > 0, Z >= 1, A > 0, ppc >= 1");
    const double cpl = b->cfg.cells_per_lambda;
    if (!(std::isfinite(x0_lambda) && std::isfinite(thickness_lambda)))
        return fail(b, PIC_ERR_INVALID_ARG, "foil position and thickness must be finite");
    const long long c0 = std::llround(x0_lambda * cpl), nc = std::llround(thickness_lambda * cpl);
    if (c0 < 0 || nc < 1 || c0 + nc > r.Nx)
        return fail(b, PIC_ERR_INVALID_ARG, "foil must lie inside the box and span at least one cell");
    const long long n = nc * static_cast<long long>(ppc);
    if (n > 2147483647LL - 64) return fail(b, PIC_ERR_INVALID_ARG, "more than 2^31 particles per species");
    const size_t mark = r.mem.size();
    pic_status st = alloc_species(b, r, 0, n);
    if (st == PIC_OK) st = alloc_species(b, r, 1, n);
    if (st != PIC_OK) {
        free_from(b, r.mem, mark);
        clear_species(r, 0);
        clear_species(r, 1);
        return st;
    }
    // loaded particles go to the buffer the batch's kernels read at their first step
    launch_foil(r.dev.sp[0][b->cur], r.dev.sp[1][b->cur], static_cast<int>(c0), static_cast<int>(nc), ppc, r.seed,
                b->stream);
    b->launches++;
    HostSpecies& el = r.sp[0];
    HostSpecies& io = r.sp[1];
    el.q = -1.0;
    el.m = 1.0;
    el.w = ne_over_nc / ppc;
    io.q = ion_Z;
    io.m = (ion_Z == 1 && ion_A == 1.0) ? kMpMe : ion_A * kMuMe;
    io.w = ne_over_nc / (static_cast<double>(ion_Z) * ppc);
    el.loaded = io.loaded = true;
    return PIC_OK;
}

// Upload host particle arrays (already in cell order) into the load buffer.
pic_status run_upload(Batch* b, RunHost& r, int s, int64_t n, const int32_t* cell, const float* off, const float* px,
                      const float* py, const float* pz, const int32_t* id, double w, double q, double m) {
    const size_t mark = r.mem.size();
    pic_status st = alloc_species(b, r, s, n);
    if (st != PIC_OK) {
        free_from(b, r.mem, mark);
        clear_species(r, s);
        return st;
    }
    const DevSpecies& d = r.dev.sp[s][b->cur];
    const size_t b4 = static_cast<size_t>(n) * 4;
    cudaError_t e = cudaSuccess;
    if (n > 0) {
        e = cudaMemcpyAsync(d.cell, cell, b4, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d.off, off, b4, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d.px, px, b4, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d.py, py, b4, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d.pz, pz, b4, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) {
            if (id) {
                e = cudaMemcpyAsync(d.id, id, b4, cudaMemcpyHostToDevice, b->stream);
            } else {
                launch_iota(d.id, n, b->stream);
                b->launches++;
            }
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // host arrays may be released after return
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        free_from(b, r.mem, mark);
        clear_species(r, s);
        return cuda_fail(b, e, "upload particles");
    }
    r.sp[s].w = w;
    r.sp[s].q = q;
    r.sp[s].m = m;
    r.sp[s].loaded = true;
    return PIC_OK;
}

pic_status check_species_args(Batch* b, RunHost& r, int species, int64_t n, double weight, double charge,
                              double mass) {
    if (species != PIC_ELECTRON && species != PIC_ION) return fail(b, PIC_ERR_INVALID_ARG, "bad species");
    if (r.started) return fail(b, PIC_ERR_STATE, "load_particles after the first step");
    if (r.sp[species].loaded) return fail(b, PIC_ERR_STATE, "species already loaded");
    if (n < 0 || n > 2147483647LL - 64) return fail(b, PIC_ERR_INVALID_ARG, "n must be in [0, 2^31 - 64]");
    if (!(mass > 0.0) || !std::isfinite(weight) || !std::isfinite(charge))
        return fail(b, PIC_ERR_INVALID_ARG, "mass must be > 0, weight and charge finite");
    return PIC_OK;
}

pic_status run_load_particles_f32(Batch* b, int id, int species, int64_t n, const int32_t* cell, const float* off,
                                  const float* px, const float* py, const float* pz, double weight, double charge,
                                  double mass) {
    RunHost& r = b->runs[id];
    pic_status st = check_species_args(b, r, species, n, weight, charge, mass);
    if (st != PIC_OK) return st;
    if (n > 0 && (!cell || !off || !px || !py || !pz)) return fail(b, PIC_ERR_INVALID_ARG, "NULL array");
    // upload as given, then check on the device: ranges, finiteness and cell order
    st = run_upload(b, r, species, n, cell, off, px, py, pz, nullptr, weight, charge, mass);
    if (st != PIC_OK || n == 0) return st;
    unsigned long long chk[3] = {0, 0, 0};
    {
        const DevSpecies& d = r.dev.sp[species][b->cur];
        PIC_CK(b, cudaMemsetAsync(b->snap_out, 0, 4 * sizeof(unsigned long long), b->stream));
        launch_validate(d.cell, d.off, d.px, d.py, d.pz, n, r.Nx, b->snap_out, b->stream);
        b->launches++;
        PIC_CK(b, cudaMemcpyAsync(chk, b->snap_out, sizeof(chk), cudaMemcpyDeviceToHost, b->stream));
        PIC_CK(b, cudaStreamSynchronize(b->stream));
    }
    if (chk[0] == 0 && chk[1] == 0 && chk[2] == 0) return PIC_OK;
    // not usable as uploaded: release it (the species stays unloaded)
    {
        std::vector<std::pair<void*, size_t>> keep;
        for (auto& a : r.mem) {
            bool mine = false;
            for (int x = 0; x < 2; ++x) {
                const DevSpecies& d = r.dev.sp[species][x];
                for (const void* q : {static_cast<const void*>(d.cell), static_cast<const void*>(d.off),
                                      static_cast<const void*>(d.px), static_cast<const void*>(d.py),
                                      static_cast<const void*>(d.pz), static_cast<const void*>(d.id)})
                    mine = mine || a.first == q;
            }
            if (mine) {
                cudaFreeAsync(a.first, b->stream);
                b->bytes -= a.second;
            } else {
                keep.push_back(a);
            }
        }
        r.mem.swap(keep);
        clear_species(r, species);
    }
    if (chk[0]) return fail(b, PIC_ERR_INVALID_ARG, "cell out of [0, Nx)");
    if (chk[1]) return fail(b, PIC_ERR_INVALID_ARG, "offset out of [0, 1) or non-finite momentum");
    // units need cell order: stable sort on the host; ids keep the load order
    std::vector<int64_t> order(static_cast<size_t>(n));
    for (int64_t i = 0; i < n; ++i) order[static_cast<size_t>(i)] = i;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t c) { return cell[a] < cell[c]; });
    std::vector<int32_t> hc(static_cast<size_t>(n)), hid(static_cast<size_t>(n));
    std::vector<float> ho(static_cast<size_t>(n)), hx(static_cast<size_t>(n)), hy(static_cast<size_t>(n)),
        hz(static_cast<size_t>(n));
    for (int64_t j = 0; j < n; ++j) {
        const int64_t i = order[static_cast<size_t>(j)];
        hc[j] = cell[i];
        ho[j] = off[i];
        hx[j] = px[i];
        hy[j] = py[i];
        hz[j] = pz[i];
        hid[j] = static_cast<int32_t>(i);
    }
    return run_upload(b, r, species, n, hc.data(), ho.data(), hx.data(), hy.data(), hz.data(), hid.data(), weight,
                      charge, mass);
}

pic_status run_inject_laser(Batch* b, int id, double a0, int polarization, int envelope, double duration_periods,
                            double rise_periods) {
    RunHost& r = b->runs[id];
    if (r.started) return fail(b, PIC_ERR_STATE, "inject_laser after the first step");
    if (r.laser_set) return fail(b, PIC_ERR_STATE, "laser already set");
    if (!(a0 >= 0.0 && std::isfinite(a0))) return fail(b, PIC_ERR_INVALID_ARG, "a0 must be finite and >= 0");
    if (polarization != PIC_LP && polarization != PIC_CP) return fail(b, PIC_ERR_INVALID_ARG, "bad polarization");
    if (envelope != PIC_ENV_SIN2 && envelope != PIC_ENV_TRAPEZOID)
        return fail(b, PIC_ERR_INVALID_ARG, "bad envelope");
    if (!(duration_periods > 0.0 && std::isfinite(duration_periods)))
        return fail(b, PIC_ERR_INVALID_ARG, "duration must be > 0");
    if (envelope == PIC_ENV_TRAPEZOID && !(rise_periods > 0.0 && 2.0 * rise_periods <= duration_periods))
        return fail(b, PIC_ERR_INVALID_ARG, "trapezoid needs 0 < 2 rise <= duration");
    r.laser.on = 1;
    r.laser.pol = polarization;
    r.laser.env = envelope;
    r.laser.a0 = a0;
    r.laser.tau = duration_periods * 2.0 * kPi;
    r.laser.rise = rise_periods * 2.0 * kPi;
    r.laser_set = true;
    return PIC_OK;
}

pic_status run_set_fields(Batch* b, int id, const double* const* src) {
    RunHost& r = b->runs[id];
    if (r.started) return fail(b, PIC_ERR_STATE, "set_fields after the first step");
    if (r.fields_set) return fail(b, PIC_ERR_STATE, "fields already set");
    std::vector<float> h(r.glen);
    for (int c = 0; c < 5; ++c) {
        std::fill(h.begin(), h.end(), 0.0f);
        const int n = (c == 1 || c == 2) ? r.Nx + 1 : r.Nx;
        if (src[c])
            for (int i = 0; i < n; ++i) {
                if (!std::isfinite(src[c][i])) return fail(b, PIC_ERR_INVALID_ARG, "non-finite field value");
                h[PADF + i] = static_cast<float>(src[c][i]);
            }
        // a run's fields start in buffer 0 (its parity offset makes that current)
        PIC_CK(b, cudaMemcpyAsync(r.dev.F[0][c], h.data(), r.glen * 4, cudaMemcpyHostToDevice, b->stream));
        PIC_CK(b, cudaStreamSynchronize(b->stream));
    }
    r.fields_set = true;
    return PIC_OK;
}

// Fixed-point scales and per-species constants of a run, frozen at its first step.
void finalize_run_params(Batch* b, RunHost& r) {
    RunDev& d = r.dev;
    double bound = 0.0;
    for (int s = 0; s < 2; ++s) {
        const HostSpecies& h = r.sp[s];
        d.n[s] = h.loaded ? static_cast<int32_t>(h.n) : 0;
        d.qm[s] = h.loaded ? static_cast<float>(h.q / h.m) : 0.f;
        d.qw[s] = h.loaded ? static_cast<float>(h.q * h.w) : 0.f;
        d.rad_w[s] = h.loaded ? static_cast<float>(h.w * b->dx * h.m) : 0.f;
        if (h.loaded) bound += static_cast<double>(h.n) * std::fabs(h.q * h.w) / b->cfl;
    }
    // every partial sum of the current is bounded by `bound`: keep bound * 2^fp below 2^61
    int fp = 40;
    if (bound > 0.0) fp = static_cast<int>(std::floor(61.0 - std::log2(bound)));
    r.fp_bits = std::max(8, std::min(52, fp));
    d.fp_inv = std::ldexp(1.0f, -r.fp_bits);
    for (int s = 0; s < 2; ++s) {
        // a lane's running record merges at most the 4 particles of one 16-byte slot
        // (records are flushed at the end of every round); with a margin of 4 the
        // bound below takes 16 particles of one lane over 32 lanes, each value
        // bounded by |q w| max(1, 1/cfl), and keeps every lane below 2^26
        const double vmax = r.sp[s].loaded ? std::fabs(r.sp[s].q * r.sp[s].w) * std::max(1.0, 1.0 / b->cfl) : 0.0;
        int ls = 40;
        if (vmax > 0.0) ls = static_cast<int>(std::floor(26.0 - std::log2(16.0 * vmax)));
        ls = std::min(ls, r.fp_bits);
        d.lscale[s] = std::ldexp(1.0f, ls);
        d.lshift[s] = std::min(62, r.fp_bits - ls);
    }
    d.rr = r.rr;
}

// Grow the batch-level unit table and sort scratch to hold `need` units.
pic_status ensure_units(Batch* b, int need) {
    if (need <= b->max_units) return PIC_OK;
    const int mu = std::max(need, b->max_units + b->max_units / 2);
    std::vector<std::pair<void*, size_t>> fresh;
    UnitTable u{};
    double* rp = nullptr;
    int32_t *cn = nullptr, *of = nullptr;
    const size_t m = static_cast<size_t>(mu);
    pic_status st = PIC_OK;
    if (st == PIC_OK) st = dalloc_t(b, fresh, &u.run, m);
    if (st == PIC_OK) st = dalloc_t(b, fresh, &u.species, m);
    if (st == PIC_OK) st = dalloc_t(b, fresh, &u.start, m);
    if (st == PIC_OK) st = dalloc_t(b, fresh, &u.end, m);
    if (st == PIC_OK) st = dalloc_t(b, fresh, &u.lo, m);
    if (st == PIC_OK) st = dalloc_t(b, fresh, &u.hi, m);
    if (st == PIC_OK) st = dalloc_t(b, fresh, &u.count, 4);
    if (st == PIC_OK) st = dalloc_t(b, fresh, &rp, m);
    if (st == PIC_OK) st = dalloc_t(b, fresh, &cn, m * SSTR);
    if (st == PIC_OK) st = dalloc_t(b, fresh, &of, m * SSTR);
    if (st != PIC_OK) {
        free_all(b, fresh);
        return st;
    }
    // the unit table is rebuilt right after every growth (the radiated partials
    // were flushed by the sort that preceded it)
    for (void* p : {static_cast<void*>(b->units.run), static_cast<void*>(b->units.species),
                    static_cast<void*>(b->units.start), static_cast<void*>(b->units.end),
                    static_cast<void*>(b->units.lo), static_cast<void*>(b->units.hi),
                    static_cast<void*>(b->units.count), static_cast<void*>(b->rad_part), static_cast<void*>(b->cnt),
                    static_cast<void*>(b->offs)})
        free_one(b, p);
    for (auto& f : fresh) b->mem.push_back(f);
    b->units = u;
    b->rad_part = rp;
    b->cnt = cn;
    b->offs = of;
    b->max_units = mu;
    b->epoch++;
    return PIC_OK;
}

SortParams sort_params(Batch* b) {
    SortParams S{};
    S.runs = b->d_runs;
    S.nruns = b->max_runs;
    S.units = b->units;
    S.cnt = b->cnt;
    S.offs = b->offs;
    S.rs_units = b->rs_units;
    S.status = b->d_status;
    S.k = b->since_sort;
    S.cur = b->cur;
    S.max_units = b->max_units;
    int mx = 1;
    for (auto& r : b->runs)
        if (r.used) mx = std::max(mx, r.Nx);
    S.kb_max = (mx + KEY_T - 1) / KEY_T;
    S.unit_p = b->unit_p;
    return S;
}

// Upload the run table (pointers, constants, active flags).
pic_status upload_table(Batch* b) {
    if (!b->table_dirty) return PIC_OK;
    for (int i = 0; i < b->max_runs; ++i) {
        const RunHost& r = b->runs[i];
        if (!r.used) {
            std::memset(&b->h_runs[i], 0, sizeof(RunDev));
            continue;
        }
        RunDev d = r.dev;
        d.active = r.active ? 1 : 0;
        b->h_runs[i] = d;
    }
    PIC_CK(b, cudaMemcpyAsync(b->d_runs, b->h_runs, sizeof(RunDev) * b->max_runs, cudaMemcpyHostToDevice,
                              b->stream));
    PIC_CK(b, cudaStreamSynchronize(b->stream));  // the pinned staging is rewritten by the next upload
    b->table_dirty = false;
    return PIC_OK;
}

// Block table of the Yee kernel: FIELD_NODES nodes of one active run per block.
pic_status upload_blocks(Batch* b) {
    if (!b->layout_dirty) return PIC_OK;
    std::vector<int32_t> br, bi;
    for (int i = 0; i < b->max_runs; ++i) {
        const RunHost& r = b->runs[i];
        if (!r.used || !r.active) continue;
        for (int i0 = 0; i0 <= r.Nx; i0 += FIELD_NODES) {
            br.push_back(i);
            bi.push_back(i0);
        }
    }
    const int n = static_cast<int>(br.size());
    if (n > b->blk_cap) {
        std::vector<std::pair<void*, size_t>> fresh;
        int32_t *a = nullptr, *c = nullptr;
        pic_status st = dalloc_t(b, fresh, &a, static_cast<size_t>(n));
        if (st == PIC_OK) st = dalloc_t(b, fresh, &c, static_cast<size_t>(n));
        if (st != PIC_OK) {
            free_all(b, fresh);
            return st;
        }
        free_one(b, b->d_blk_run);
        free_one(b, b->d_blk_i0);
        for (auto& f : fresh) b->mem.push_back(f);
        b->d_blk_run = a;
        b->d_blk_i0 = c;
        b->blk_cap = n;
    }
    if (n > 0) {
        PIC_CK(b, cudaMemcpyAsync(b->d_blk_run, br.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, b->stream));
        PIC_CK(b, cudaMemcpyAsync(b->d_blk_i0, bi.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, b->stream));
        PIC_CK(b, cudaStreamSynchronize(b->stream));
    }
    b->nblk = n;
    b->layout_dirty = false;
    b->epoch++;  // the Yee grid, and possibly the sort's, changed shape
    return PIC_OK;
}

void rad_flush(Batch* b, cudaStream_t st) {
    if (b->max_units == 0) return;
    launch_rad_flush(b->d_runs, b->max_runs, b->rs_units, b->rad_part, st);
    b->launches++;
}
void rad_flush(Batch* b) { rad_flush(b, b->stream); }

void do_sort(Batch* b) {
    SortParams S = sort_params(b);
    int nl = 0;
    {
        Timed t(b, 2);
        rad_flush(b);
        launch_sort(S, b->stream, &nl);
    }
    b->launches += nl;
    b->cur ^= 1;
    b->sorts++;
    b->since_sort = 0;
}

// Start runs that have not stepped yet.  They join at a sort boundary, so
// that every active run's particles are sorted when the unit table is rebuilt
// (their own particles were loaded in cell order into the current buffer).
pic_status activate_pending(Batch* b) {
    bool any = false;
    for (auto& r : b->runs)
        if (r.used && !r.started) any = true;
    if (!any) return PIC_OK;
    pic_status st = upload_table(b);  // the sort below reads the device run table
    if (st != PIC_OK) return st;
    if (b->since_sort > 0) {
        do_sort(b);
        // runs loaded before this sort have their particles in the old buffer
        for (auto& r : b->runs)
            if (r.used && !r.started)
                for (int s = 0; s < 2; ++s) std::swap(r.dev.sp[s][0], r.dev.sp[s][1]);
    }
    // units the active and the joining runs can need (each tile adds at most one partial unit)
    int64_t need = 1;
    std::vector<int> joining;
    for (int i = 0; i < b->max_runs; ++i) {
        const RunHost& r = b->runs[i];
        if (!r.used || r.finished || (r.started && !r.active)) continue;
        if (!r.started) joining.push_back(i);
        const int ntiles = (r.Nx + TILE - 1) / TILE;
        for (int s = 0; s < 2; ++s)
            if (r.sp[s].loaded) need += (r.sp[s].n + b->unit_p - 1) / b->unit_p + ntiles + 1;
    }
    if (need > (1 << 30)) return fail(b, PIC_ERR_INVALID_ARG, "too many work units");
    st = ensure_units(b, static_cast<int>(need));
    if (st != PIC_OK) return st;  // the joining runs stay pending
    for (int i : joining) {
        RunHost& r = b->runs[i];
        finalize_run_params(b, r);
        r.started = true;
        r.active = true;
        r.admit_step = b->gstep;
        r.dev.fpar = static_cast<int>(b->gstep & 1);  // buffer 0 is current at the first step
    }
    b->table_dirty = b->layout_dirty = true;
    st = upload_blocks(b);
    if (st != PIC_OK) {
        for (int i : joining) b->runs[i].started = b->runs[i].active = false;
        return st;
    }
    if ((st = upload_table(b)) != PIC_OK) return st;
    SortParams S = sort_params(b);
    int nl = 0;
    launch_build_units(S, b->stream, &nl);
    b->launches += nl;
    return PIC_OK;
}

void deactivate(Batch* b, int id) {
    RunHost& r = b->runs[id];
    r.active = false;
    r.finished = true;
    r.pbuf = b->cur;
    r.fbuf = static_cast<int>((b->gstep + r.dev.fpar) & 1);
    b->table_dirty = b->layout_dirty = true;
}

// Laser source values of the coming `steps` steps for every active run,
// uploaded through a pinned ring: step j of the chunk reads d_inc + j * 6 * max_runs.
pic_status upload_incident(Batch* b, int steps) {
    const size_t per_step = static_cast<size_t>(6) * b->max_runs;
    float* h = b->h_inc + static_cast<size_t>(b->inc_slot) * per_step * KMAX;
    PIC_CK(b, cudaEventSynchronize(b->inc_ev[b->inc_slot]));
    for (int j = 0; j < steps; ++j) {
        float* hj = h + j * per_step;
        for (int i = 0; i < b->max_runs; ++i) {
            const RunHost& r = b->runs[i];
            if (!r.used || !r.active) continue;
            const double tn = static_cast<double>(b->gstep + j - r.admit_step + r.t_offset) * b->dt;
            const double ts[3] = {tn, tn + 0.5 * b->dt + 0.5 * b->dx, tn + b->dt};
            for (int k = 0; k < 3; ++k) incident(r.laser, ts[k], &hj[6 * i + 2 * k], &hj[6 * i + 2 * k + 1]);
        }
    }
    PIC_CK(b, cudaMemcpyAsync(b->d_inc, h, sizeof(float) * per_step * steps, cudaMemcpyHostToDevice, b->stream));
    cudaEventRecord(b->inc_ev[b->inc_slot], b->stream);
    b->inc_slot = (b->inc_slot + 1) % kIncRing;
    return PIC_OK;
}

PushParams push_params(const Batch* b, int64_t gstep, int k, int cur) {
    PushParams P{};
    P.runs = b->d_runs;
    P.units = b->units;
    P.rad_part = b->rad_part;
    P.status = b->d_status;
    P.gstep = gstep;
    P.k = k;
    P.cur = cur;
    P.cfl = static_cast<float>(b->cfl);
    P.dt = static_cast<float>(b->dt);
    P.eps = static_cast<float>(b->eps);
    return P;
}

FieldParams field_params(const Batch* b, int64_t gstep, int j) {
    FieldParams Q{};
    Q.runs = b->d_runs;
    Q.blk_run = b->d_blk_run;
    Q.blk_i0 = b->d_blk_i0;
    Q.inc = b->d_inc + static_cast<size_t>(j) * 6 * b->max_runs;
    Q.gstep = gstep;
    Q.dt = b->dt;
    Q.c = static_cast<float>(b->cfl);
    Q.hc = static_cast<float>(0.5 * b->cfl);
    Q.fdt = static_cast<float>(b->dt);
    return Q;
}

// The graph of one sort interval starting at step parity par0 with current
// particle buffer cur (captured on the batch's capture stream, then reused).
pic_status chunk_graph(Batch* b, int par0, int cur, cudaGraphExec_t* out) {
    cudaGraphExec_t& ex = b->graph[par0][cur];
    if (ex && b->graph_epoch[par0][cur] == b->epoch && b->graph_timed[par0][cur] == b->timing) {
        *out = ex;
        return PIC_OK;
    }
    drop_graph(b, par0, cur);
    const int I = b->sort_interval;
    cudaStream_t cs = b->cap_stream;
    std::vector<EventPair>& ev = b->graph_ev[par0][cur];
    // timing on: an event-record node before and after each timed launch
    auto mark = [&](int kind, bool open) {
        if (!b->timing) return;
        if (open) ev.push_back(EventPair{take_event(b), take_event(b), kind});
        cudaEventRecordWithFlags(open ? ev.back().a : ev.back().b, cs, cudaEventRecordExternal);
    };
    PIC_CK(b, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    for (int j = 0; j < I; ++j) {
        mark(0, true);
        launch_push(push_params(b, par0 + j, j, cur), b->max_units, b->slot_w, cs);
        mark(0, false);
        mark(1, true);
        launch_field(field_params(b, par0 + j, j), b->nblk, cs);
        mark(1, false);
    }
    mark(2, true);
    launch_rad_flush(b->d_runs, b->max_runs, b->rs_units, b->rad_part, cs);
    SortParams S = sort_params(b);
    S.k = I;
    S.cur = cur;
    int nl = 0;
    launch_sort(S, cs, &nl);
    mark(2, false);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        ex = nullptr;
        return cuda_fail(b, e, "chunk graph");
    }
    b->graph_epoch[par0][cur] = b->epoch;
    b->graph_timed[par0][cur] = b->timing;
    *out = ex;
    return PIC_OK;
}

pic_status batch_step(Batch* b, int64_t n, int64_t* done) {
    if (done) *done = 0;
    pic_status st = activate_pending(b);
    if (st != PIC_OK) return st;
    if ((st = upload_table(b)) != PIC_OK) return st;
    if ((st = upload_blocks(b)) != PIC_OK) return st;
    const int I = b->sort_interval;
    int64_t it = 0;
    // laser source values of the single steps below, uploaded for up to KMAX
    // steps at a time (one copy instead of one per step); a graph launch
    // uploads its own interval over them
    int inc_pos = 0, inc_len = 0;
    while (it < n) {
        int nact = 0;
        bool whole_chunk = b->graphs_on && b->since_sort == 0 && n - it >= I;
        for (auto& r : b->runs) {
            if (!r.used || !r.active) continue;
            nact++;
            if (r.steps_target > 0 && r.steps_target - r.steps_done < I) whole_chunk = false;
        }
        if (nact == 0) break;
        if (whole_chunk) {
            // a whole sort interval as one graph launch; no run ends before its last step
            cudaGraphExec_t ex = nullptr;
            const int gp = static_cast<int>(b->gstep & 1), gc = b->cur;
            if ((st = chunk_graph(b, gp, gc, &ex)) != PIC_OK) return st;
            if ((st = upload_incident(b, I)) != PIC_OK) return st;
            inc_pos = inc_len = 0;
            read_graph_timing(b, gp, gc);  // its previous launch (two chunks ago), before its events are reused
            PIC_CK(b, cudaGraphLaunch(ex, b->stream));
            b->graph_unread[gp][gc] = b->timing;
            b->graph_launches++;
            b->launches += 2 * I + 1 + 8;
            b->push_launches += I;
            b->gstep += I;
            b->cur ^= 1;
            b->sorts++;
            it += I;
            bool ended = false;
            for (auto& r : b->runs) {
                if (!r.used || !r.active) continue;
                r.steps_done += I;
                if (r.steps_target > 0 && r.steps_done >= r.steps_target) ended = true;
            }
            if (ended) {  // runs that end with this chunk: sorted and flushed by it
                for (int i = 0; i < b->max_runs; ++i) {
                    RunHost& r = b->runs[i];
                    if (r.used && r.active && r.steps_target > 0 && r.steps_done >= r.steps_target) deactivate(b, i);
                }
                if ((st = upload_table(b)) != PIC_OK) return st;
                if ((st = upload_blocks(b)) != PIC_OK) return st;
            }
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(b, e, "chunk launch");
            continue;
        }
        if (inc_pos >= inc_len) {
            inc_len = static_cast<int>(std::min<int64_t>(n - it, KMAX));
            inc_pos = 0;
            if ((st = upload_incident(b, inc_len)) != PIC_OK) return st;
        }
        {
            Timed t(b, 0);
            launch_push(push_params(b, b->gstep, b->since_sort, b->cur), b->max_units, b->slot_w, b->stream);
        }
        {
            Timed t(b, 1);
            launch_field(field_params(b, b->gstep, inc_pos++), b->nblk, b->stream);
        }
        b->launches += 2;
        b->push_launches++;
        b->gstep++;
        b->since_sort++;
        bool ended = false;
        for (auto& r : b->runs) {
            if (!r.used || !r.active) continue;
            r.steps_done++;
            if (r.steps_target > 0 && r.steps_done >= r.steps_target) ended = true;
        }
        // a run that ends on a sort step is sorted first, as it would be alone
        if (b->since_sort >= b->sort_interval) do_sort(b);
        if (ended) {
            if (b->since_sort > 0) rad_flush(b);  // finished runs take their radiated energy with them
            for (int i = 0; i < b->max_runs; ++i) {
                RunHost& r = b->runs[i];
                if (r.used && r.active && r.steps_target > 0 && r.steps_done >= r.steps_target) deactivate(b, i);
            }
            if ((st = upload_table(b)) != PIC_OK) return st;
            if ((st = upload_blocks(b)) != PIC_OK) return st;
        }
        if ((it & 255) == 255) {
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(b, e, "step launch");
        }
        ++it;
    }
    if (it > 0 && b->since_sort > 0) rad_flush(b);
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(b, e, "step");
    collect_timing(b);
    read_all_graph_timing(b);
    int hst = 0;
    PIC_CK(b, cudaMemcpy(&hst, b->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (done) *done = it;
    if (hst & ST_TIMEOUT) return fail(b, PIC_ERR_TIMEOUT, "a bounded device wait (TMA field window) gave up");
    if (hst & ST_WINDOW) return fail(b, PIC_ERR_STATE, "a particle left its unit window");
    return PIC_OK;
}

// Units a batch can need with unit size unit_p (each tile adds at most one
// partial unit; merged groups only lower the count).
int64_t units_needed(const Batch* b, int unit_p) {
    int64_t need = 1;
    for (const auto& r : b->runs) {
        if (!r.used || !r.active) continue;
        const int ntiles = (r.Nx + TILE - 1) / TILE;
        for (int s = 0; s < 2; ++s)
            if (r.sp[s].loaded) need += (r.sp[s].n + unit_p - 1) / unit_p + ntiles + 1;
    }
    return need;
}

// Set the launch shapes: work-unit size (takes effect through a sort now, which
// rebuilds the unit table) and sort interval.
pic_status set_shapes(Batch* b, int unit_p, int interval, int slot_w) {
    if (unit_p < UNIT_P_MIN || unit_p > UNIT_P_MAX || (unit_p & (unit_p - 1)) != 0)
        return fail(b, PIC_ERR_INVALID_ARG, "unit size must be a power of two in [1024, 16384]");
    if (slot_w != 2 && slot_w != 4) return fail(b, PIC_ERR_INVALID_ARG, "particles per thread must be 2 or 4");
    if (interval < 1 || interval > KMAX) return fail(b, PIC_ERR_INVALID_ARG, "sort interval must be in [1, 96]");
    pic_status st = activate_pending(b);
    if (st != PIC_OK) return st;
    bool any = false;
    for (auto& r : b->runs) any = any || (r.used && r.active);
    if (unit_p != b->unit_p) {
        // sort with the current table first (it also flushes the radiated
        // partials), then rebuild the table from the sorted cells with the new size
        if (any && b->since_sort > 0) do_sort(b);
        const int64_t need = units_needed(b, unit_p);
        if (need > (1 << 30)) return fail(b, PIC_ERR_INVALID_ARG, "too many work units");
        if ((st = ensure_units(b, static_cast<int>(need))) != PIC_OK) return st;
        b->unit_p = unit_p;
        if (any) {
            SortParams S = sort_params(b);
            int nl = 0;
            launch_build_units(S, b->stream, &nl);
            b->launches += nl;
        }
    }
    if (interval != b->sort_interval && b->since_sort > 0) do_sort(b);
    b->sort_interval = interval;
    b->slot_w = slot_w;
    b->epoch++;  // recapture the step graphs (interval, kernel variant)
    return PIC_OK;
}

// Shape tuner: step the batch for a trial at each candidate work-unit size
// (at the current sort interval), keep the fastest, then at each candidate
// sort interval.  Each trial runs whole sort intervals as CUDA graphs after
// one warm-up interval and measures the wall time per step.  The trial steps
// are real steps of every active run; the shapes change only the order of
// single-precision sums.
pic_status tune_shapes(Batch* b, int64_t steps_per, int* unit_out, int* interval_out, int* slot_out,
                       double* ms_out) {
    static const int slots[2] = {4, 2};
    static const int units[4] = {2048, 4096, 8192, 16384};
    static const int cand[5] = {8, 16, 32, 64, 96};
    if (steps_per < 1) return fail(b, PIC_ERR_INVALID_ARG, "steps_per_candidate must be >= 1");
    if (b->timing) return fail(b, PIC_ERR_STATE, "turn timing off before tuning");
    if (ms_out)
        for (int i = 0; i < 11; ++i) ms_out[i] = -1.0;
    auto trial = [&](int unit_p, int interval, int slot_w, double* per) -> pic_status {
        *per = -1.0;
        bool any = false;
        for (auto& r : b->runs) any = any || (r.used && r.active);
        if (!any) return PIC_OK;
        pic_status st = set_shapes(b, unit_p, interval, slot_w);
        if (st != PIC_OK) return st;
        int64_t done = 0;
        if ((st = batch_step(b, interval, &done)) != PIC_OK) return st;  // captures the shape's graphs
        if (done < interval) return PIC_OK;
        const int64_t n = std::max<int64_t>(interval, steps_per / interval * interval);
        const auto t0 = std::chrono::steady_clock::now();
        if ((st = batch_step(b, n, &done)) != PIC_OK) return st;
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (done == n) *per = ms / static_cast<double>(n);  // else a run ended inside the trial
        return PIC_OK;
    };
    pic_status st = activate_pending(b);
    if (st != PIC_OK) return st;
    int best_w = b->slot_w, best_u = b->unit_p, best_i = b->sort_interval;
    double best = 1e300;
    for (int c = 0; c < 2; ++c) {
        double per;
        if ((st = trial(best_u, best_i, slots[c], &per)) != PIC_OK) return st;
        if (ms_out) ms_out[c] = per;
        if (per > 0.0 && per < best) {
            best = per;
            best_w = slots[c];
        }
    }
    best = 1e300;
    for (int c = 0; c < 4; ++c) {
        double per;
        if ((st = trial(units[c], best_i, best_w, &per)) != PIC_OK) return st;
        if (ms_out) ms_out[2 + c] = per;
        if (per > 0.0 && per < best) {
            best = per;
            best_u = units[c];
        }
    }
    best = 1e300;
    for (int c = 0; c < 5; ++c) {
        double per;
        if ((st = trial(best_u, cand[c], best_w, &per)) != PIC_OK) return st;
        if (ms_out) ms_out[6 + c] = per;
        if (per > 0.0 && per < best) {
            best = per;
            best_i = cand[c];
        }
    }
    if (best >= 1e300) return fail(b, PIC_ERR_STATE, "no active run stepped through a whole trial");
    if ((st = set_shapes(b, best_u, best_i, best_w)) != PIC_OK) return st;
    if (unit_out) *unit_out = best_u;
    if (interval_out) *interval_out = best_i;
    if (slot_out) *slot_out = best_w;
    return PIC_OK;
}

// particle buffer and field buffer holding a run's current state
int run_pbuf(const Batch* b, const RunHost& r) { return r.finished ? r.pbuf : b->cur; }
int run_fbuf(const Batch* b, const RunHost& r) {
    if (r.finished) return r.fbuf;
    if (!r.started) return 0;
    return static_cast<int>((b->gstep + r.dev.fpar) & 1);
}

pic_status run_energy(Batch* b, int id, double out[6]) {
    const RunHost& r = b->runs[id];
    DiagParams D{};
    const int fb = run_fbuf(b, r);
    for (int c = 0; c < 5; ++c) D.F[c] = r.dev.F[fb][c];
    D.Nx = r.Nx;
    D.is = r.is;
    D.hc = static_cast<float>(0.5 * b->cfl);
    int nb = launch_field_energy(D, b->diag_partials, kMaxDiagBlocks, b->stream);
    launch_reduce_partials(b->diag_partials, nb, b->dx, b->diag_out + 0, b->stream);
    b->launches += 2;
    for (int s = 0; s < 2; ++s) {
        const HostSpecies& h = r.sp[s];
        if (!h.loaded || h.n == 0) {
            PIC_CK(b, cudaMemsetAsync(b->diag_out + 1 + s, 0, sizeof(double), b->stream));
            continue;
        }
        nb = launch_kinetic(r.dev.sp[s][run_pbuf(b, r)], h.n, b->diag_partials, kMaxDiagBlocks, b->stream);
        launch_reduce_partials(b->diag_partials, nb, h.w * b->dx * h.m, b->diag_out + 1 + s, b->stream);
        b->launches += 2;
    }
    double d[3], t[3];
    PIC_CK(b, cudaMemcpyAsync(d, b->diag_out, sizeof(d), cudaMemcpyDeviceToHost, b->stream));
    PIC_CK(b, cudaMemcpyAsync(t, r.dev.tally, sizeof(t), cudaMemcpyDeviceToHost, b->stream));
    PIC_CK(b, cudaStreamSynchronize(b->stream));
    out[0] = d[0];
    out[1] = d[1];
    out[2] = d[2];
    out[3] = t[0];
    out[4] = t[1];
    out[5] = t[2];
    return PIC_OK;
}

pic_status run_spectra(Batch* b, int id, int species, int nbins, double e_min, double e_max, double* counts,
                       double* radiated) {
    if (species != PIC_ELECTRON && species != PIC_ION) return fail(b, PIC_ERR_INVALID_ARG, "bad species");
    if (nbins < 1 || nbins > (1 << 24) || !counts || !(e_max > e_min) || !std::isfinite(e_min) ||
        !std::isfinite(e_max))
        return fail(b, PIC_ERR_INVALID_ARG, "need 1 <= nbins <= 2^24, e_max > e_min, counts != NULL");
    const RunHost& r = b->runs[id];
    const HostSpecies& h = r.sp[species];
    std::vector<unsigned long long> hb(static_cast<size_t>(nbins) + 2, 0ull);
    if (h.loaded && h.n > 0) {
        if (b->bins_cap < nbins + 2) {
            std::vector<std::pair<void*, size_t>> fresh;
            unsigned long long* nbp = nullptr;
            pic_status st = dalloc_t(b, fresh, &nbp, static_cast<size_t>(nbins) + 2);
            if (st != PIC_OK) return st;
            free_one(b, b->bins);
            b->mem.push_back(fresh[0]);
            b->bins = nbp;
            b->bins_cap = nbins + 2;
        }
        PIC_CK(b, cudaMemsetAsync(b->bins, 0, sizeof(unsigned long long) * (nbins + 2), b->stream));
        launch_spectrum(r.dev.sp[species][run_pbuf(b, r)], h.n, h.m * kMec2MeV, nbins, e_min, e_max, b->bins,
                        b->stream);
        b->launches++;
        PIC_CK(b, cudaMemcpyAsync(hb.data(), b->bins, sizeof(unsigned long long) * (nbins + 2),
                                  cudaMemcpyDeviceToHost, b->stream));
    }
    double tally0 = 0.0;
    PIC_CK(b, cudaMemcpyAsync(&tally0, r.dev.tally, sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    PIC_CK(b, cudaStreamSynchronize(b->stream));
    const double width = (e_max - e_min) / nbins;
    const double wdx = h.w * b->dx;
    for (int k = 0; k < nbins; ++k) counts[k] = static_cast<double>(hb[k]) * wdx / width;
    if (radiated) {
        // energy unit per area: m_e c^2 n_c (c/omega), n_c = eps0 m_e omega^2 / e^2 (SI)
        const double me = 9.1093837015e-31, c = 299792458.0, qe = 1.602176634e-19, eps0 = 8.8541878128e-12;
        const double omega = 2.0 * kPi * c / (b->cfg.lambda_um * 1e-6);
        const double nc = eps0 * me * omega * omega / (qe * qe);
        *radiated = tally0 * me * c * c * nc * c / omega;
    }
    return PIC_OK;
}

pic_status run_read_particles(Batch* b, int id, int species, int64_t cap, double* x, double* px, double* py,
                              double* pz, int32_t* flag, int64_t* nout) {
    if (species != PIC_ELECTRON && species != PIC_ION) return fail(b, PIC_ERR_INVALID_ARG, "bad species");
    const RunHost& r = b->runs[id];
    const HostSpecies& h = r.sp[species];
    const int64_t n = h.loaded ? h.n : 0;
    if (nout) *nout = n;
    if (cap <= 0 || n == 0) return PIC_OK;
    std::vector<int32_t> c(n), idv(n);
    std::vector<float> o(n), qx(n), qy(n), qz(n);
    const DevSpecies& d = r.dev.sp[species][run_pbuf(b, r)];
    const size_t by = static_cast<size_t>(n) * 4;
    PIC_CK(b, cudaMemcpyAsync(c.data(), d.cell, by, cudaMemcpyDeviceToHost, b->stream));
    PIC_CK(b, cudaMemcpyAsync(idv.data(), d.id, by, cudaMemcpyDeviceToHost, b->stream));
    PIC_CK(b, cudaMemcpyAsync(o.data(), d.off, by, cudaMemcpyDeviceToHost, b->stream));
    PIC_CK(b, cudaMemcpyAsync(qx.data(), d.px, by, cudaMemcpyDeviceToHost, b->stream));
    PIC_CK(b, cudaMemcpyAsync(qy.data(), d.py, by, cudaMemcpyDeviceToHost, b->stream));
    PIC_CK(b, cudaMemcpyAsync(qz.data(), d.pz, by, cudaMemcpyDeviceToHost, b->stream));
    PIC_CK(b, cudaStreamSynchronize(b->stream));
    for (int64_t i = 0; i < n; ++i) {
        const int64_t j = idv[i];
        if (j < 0 || j >= n) return fail(b, PIC_ERR_STATE, "corrupt particle id");
        if (j >= cap) continue;
        int fl = 0;
        double xi;
        if (c[i] < 0) {  // frozen at a wall, stored as -1 - (last cell)
            const int key = -1 - c[i];
            fl = key == 0 ? -1 : 1;
            xi = key == 0 ? 0.0 : static_cast<double>(r.Nx);
        } else {
            xi = static_cast<double>(c[i]) + o[i];
        }
        if (x) x[j] = xi * b->dx;
        if (px) px[j] = qx[i];
        if (py) py[j] = qy[i];
        if (pz) pz[j] = qz[i];
        if (flag) flag[j] = fl;
    }
    return PIC_OK;
}

// Skin-layer snapshot: d of Eq. (damping) and chi per particle on the device,
// with their maxima and the count of chi >= chi_flag; per-particle values
// (with x, p_x, p_perp) returned in load order when cap > 0.
pic_status run_snapshot(Batch* b, int id, int species, double chi_flag, int64_t cap, double* x, double* px,
                        double* pperp, double* d, double* chi, double* summary, int64_t* nout) {
    if (species != PIC_ELECTRON && species != PIC_ION) return fail(b, PIC_ERR_INVALID_ARG, "bad species");
    if (!(chi_flag >= 0.0) || !std::isfinite(chi_flag)) return fail(b, PIC_ERR_INVALID_ARG, "chi_flag must be >= 0");
    const RunHost& r = b->runs[id];
    const HostSpecies& h = r.sp[species];
    const int64_t n = h.loaded ? h.n : 0;
    if (nout) *nout = n;
    if (summary) summary[0] = summary[1] = summary[2] = 0.0;
    if (n == 0) return PIC_OK;
    const bool per = cap > 0 && (x || px || pperp || d || chi);
    std::vector<std::pair<void*, size_t>> tmp;
    float *dd = nullptr, *dc = nullptr;
    if (per) {
        pic_status st = dalloc_t(b, tmp, &dd, static_cast<size_t>(n));
        if (st == PIC_OK) st = dalloc_t(b, tmp, &dc, static_cast<size_t>(n));
        if (st != PIC_OK) {
            free_all(b, tmp);
            return st;
        }
    }
    SnapParams S{};
    const int fb = run_fbuf(b, r);
    for (int c = 0; c < 5; ++c) S.F[c] = r.dev.F[fb][c];
    S.eps = static_cast<float>(b->eps);
    S.ecr_inv = static_cast<float>(2.0 * kPi * kLambdaCUm / b->cfg.lambda_um);  // 1 / (m c^2 / hbar omega)
    S.chi_flag = static_cast<float>(chi_flag);
    const DevSpecies& sp = r.dev.sp[species][run_pbuf(b, r)];
    PIC_CK(b, cudaMemsetAsync(b->snap_out, 0, 4 * sizeof(unsigned long long), b->stream));
    launch_snapshot(sp, n, S, dd, dc, b->snap_out, b->stream);
    b->launches++;
    unsigned long long so[3];
    PIC_CK(b, cudaMemcpyAsync(so, b->snap_out, sizeof(so), cudaMemcpyDeviceToHost, b->stream));
    std::vector<int32_t> c, idv;
    std::vector<float> o, qx, qy, qz, hd, hc;
    if (per) {
        c.resize(n);
        idv.resize(n);
        o.resize(n);
        qx.resize(n);
        qy.resize(n);
        qz.resize(n);
        hd.resize(n);
        hc.resize(n);
        const size_t by = static_cast<size_t>(n) * 4;
        PIC_CK(b, cudaMemcpyAsync(c.data(), sp.cell, by, cudaMemcpyDeviceToHost, b->stream));
        PIC_CK(b, cudaMemcpyAsync(idv.data(), sp.id, by, cudaMemcpyDeviceToHost, b->stream));
        PIC_CK(b, cudaMemcpyAsync(o.data(), sp.off, by, cudaMemcpyDeviceToHost, b->stream));
        PIC_CK(b, cudaMemcpyAsync(qx.data(), sp.px, by, cudaMemcpyDeviceToHost, b->stream));
        PIC_CK(b, cudaMemcpyAsync(qy.data(), sp.py, by, cudaMemcpyDeviceToHost, b->stream));
        PIC_CK(b, cudaMemcpyAsync(qz.data(), sp.pz, by, cudaMemcpyDeviceToHost, b->stream));
        PIC_CK(b, cudaMemcpyAsync(hd.data(), dd, by, cudaMemcpyDeviceToHost, b->stream));
        PIC_CK(b, cudaMemcpyAsync(hc.data(), dc, by, cudaMemcpyDeviceToHost, b->stream));
    }
    cudaError_t e = cudaStreamSynchronize(b->stream);
    free_all(b, tmp);
    if (e != cudaSuccess) return cuda_fail(b, e, "snapshot");
    if (summary) {
        float f0, f1;
        const unsigned int u0 = static_cast<unsigned int>(so[0]), u1 = static_cast<unsigned int>(so[1]);
        std::memcpy(&f0, &u0, 4);
        std::memcpy(&f1, &u1, 4);
        summary[0] = f0;
        summary[1] = f1;
        summary[2] = static_cast<double>(so[2]);
    }
    if (!per) return PIC_OK;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t j = idv[i];
        if (j < 0 || j >= n) return fail(b, PIC_ERR_STATE, "corrupt particle id");
        if (j >= cap) continue;
        double xi;
        if (c[i] < 0) {
            const int key = -1 - c[i];
            xi = key == 0 ? 0.0 : static_cast<double>(r.Nx);
        } else {
            xi = static_cast<double>(c[i]) + o[i];
        }
        if (x) x[j] = xi * b->dx;
        if (px) px[j] = qx[i];
        if (pperp) pperp[j] = std::sqrt(static_cast<double>(qy[i]) * qy[i] + static_cast<double>(qz[i]) * qz[i]);
        if (d) d[j] = hd[i];
        if (chi) chi[j] = hc[i];
    }
    return PIC_OK;
}

// The current of a run's last step, component c (Jx, Jy, Jz), on the whole
// padded grid: its fixed-point accumulators (the set of the last step, kept
// until the next step's Yee update zeroes it) times 2^-fp.  Before the first
// step that set holds zeros, or the current a checkpoint restored into it.
pic_status last_current(Batch* b, const RunHost& r, int c, std::vector<double>& out) {
    const int lp = 1 - run_fbuf(b, r);
    std::vector<long long> h(r.glen);
    PIC_CK(b, cudaMemcpyAsync(h.data(), r.dev.J[lp][c], sizeof(long long) * r.glen, cudaMemcpyDeviceToHost,
                              b->stream));
    PIC_CK(b, cudaStreamSynchronize(b->stream));
    out.resize(r.glen);
    for (size_t i = 0; i < r.glen; ++i) out[i] = std::ldexp(static_cast<double>(h[i]), -r.fp_bits);
    return PIC_OK;
}

pic_status run_read_fields(Batch* b, int id, int comp, int64_t cap, double* out, int64_t* nout) {
    if (comp < PIC_EX || comp > PIC_JZ) return fail(b, PIC_ERR_INVALID_ARG, "bad component");
    const RunHost& r = b->runs[id];
    const bool node = comp == PIC_EY || comp == PIC_EZ || comp == PIC_JY || comp == PIC_JZ;
    const int64_t n = node ? r.Nx + 1 : r.Nx;
    if (nout) *nout = n;
    if (!out || cap < n) return fail(b, PIC_ERR_INVALID_ARG, "output too small");
    if (comp >= PIC_JX) {
        std::vector<double> j;
        pic_status st = last_current(b, r, comp - PIC_JX, j);
        if (st != PIC_OK) return st;
        for (int64_t i = 0; i < n; ++i) out[i] = j[static_cast<size_t>(PADF + i)];
        return PIC_OK;
    }
    const float* src = r.dev.F[run_fbuf(b, r)][comp];
    std::vector<float> h(static_cast<size_t>(n));
    PIC_CK(b, cudaMemcpyAsync(h.data(), src + PADF, sizeof(float) * n, cudaMemcpyDeviceToHost, b->stream));
    PIC_CK(b, cudaStreamSynchronize(b->stream));
    for (int64_t i = 0; i < n; ++i) out[i] = h[static_cast<size_t>(i)];
    return PIC_OK;
}

// ---------------------------------------------------------------------------
// checkpoint and restore of one run
// ---------------------------------------------------------------------------
constexpr char kMagic[8] = {'P', 'I', 'C', 'R', 'R', 'C', 'K', '1'};

struct CkHeader {
    char magic[8];
    int32_t version, nx, source_node, rr;
    double length_lambda, cells_per_lambda, cfl, lambda_um;
    uint64_t seed;
    int64_t steps;            // steps the run has made
    int32_t laser_on, pol, env, loaded[2];
    double a0, tau, rise;
    int64_t n[2];
    double w[2], q[2], m[2];
    double tally[4];
    int64_t glen;
};

pic_status run_save(Batch* b, int id, const char* path) {
    RunHost& r = b->runs[id];
    if (r.active && b->since_sort > 0) do_sort(b);  // saved in cell order (the sort also flushes the radiated partials)
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(b, PIC_ERR_INVALID_ARG, std::string("cannot open ") + path + " for writing");
    CkHeader h{};
    std::memcpy(h.magic, kMagic, 8);
    h.version = 1;
    h.nx = r.Nx;
    h.source_node = r.is;
    h.rr = r.rr;
    h.length_lambda = r.length_lambda;
    h.cells_per_lambda = b->cfg.cells_per_lambda;
    h.cfl = b->cfl;
    h.lambda_um = b->cfg.lambda_um;
    h.seed = r.seed;
    h.steps = r.steps_done + r.t_offset;
    h.laser_on = r.laser_set ? 1 : 0;
    h.pol = r.laser.pol;
    h.env = r.laser.env;
    h.a0 = r.laser.a0;
    h.tau = r.laser.tau;
    h.rise = r.laser.rise;
    for (int s = 0; s < 2; ++s) {
        h.loaded[s] = r.sp[s].loaded ? 1 : 0;
        h.n[s] = r.sp[s].loaded ? r.sp[s].n : 0;
        h.w[s] = r.sp[s].w;
        h.q[s] = r.sp[s].q;
        h.m[s] = r.sp[s].m;
    }
    h.glen = static_cast<int64_t>(r.glen);
    cudaError_t e = cudaMemcpyAsync(h.tally, r.dev.tally, sizeof(h.tally), cudaMemcpyDeviceToHost, b->stream);
    std::vector<char> buf;
    auto put = [&](const void* dev, size_t bytes) {
        buf.resize(bytes);
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(buf.data(), dev, bytes, cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        return e == cudaSuccess && std::fwrite(buf.data(), 1, bytes, f) == bytes;
    };
    bool ok = (e = cudaStreamSynchronize(b->stream)) == cudaSuccess && std::fwrite(&h, sizeof(h), 1, f) == 1;
    const int fb = run_fbuf(b, r), pb = run_pbuf(b, r);
    for (int c = 0; c < 5 && ok; ++c) ok = put(r.dev.F[fb][c], r.glen * 4);
    for (int c = 0; c < 3 && ok; ++c) {  // the last step's current, as float
        std::vector<double> j;
        if (last_current(b, r, c, j) != PIC_OK) {
            ok = false;
            break;
        }
        std::vector<float> jf(j.begin(), j.end());
        ok = std::fwrite(jf.data(), 4, jf.size(), f) == jf.size();
    }
    for (int s = 0; s < 2 && ok; ++s) {
        if (!h.loaded[s] || h.n[s] == 0) continue;
        const DevSpecies& d = r.dev.sp[s][pb];
        const size_t by = static_cast<size_t>(h.n[s]) * 4;
        for (const void* a : {static_cast<const void*>(d.cell), static_cast<const void*>(d.off),
                              static_cast<const void*>(d.px), static_cast<const void*>(d.py),
                              static_cast<const void*>(d.pz), static_cast<const void*>(d.id)})
            ok = ok && put(a, by);
    }
    ok = (std::fclose(f) == 0) && ok;
    if (e != cudaSuccess) return cuda_fail(b, e, "save");
    if (!ok) return fail(b, PIC_ERR_INVALID_ARG, std::string("write failed: ") + path);
    return PIC_OK;
}

// Restore into a freshly opened run slot (grid allocated, nothing loaded).
pic_status run_restore(Batch* b, int id, FILE* f, const CkHeader& h) {
    RunHost& r = b->runs[id];
    std::vector<char> buf;
    auto get = [&](void* dev, size_t bytes) -> pic_status {
        buf.resize(bytes);
        if (bytes && std::fread(buf.data(), 1, bytes, f) != bytes)
            return fail(b, PIC_ERR_INVALID_ARG, "checkpoint file is truncated");
        cudaError_t e = bytes ? cudaMemcpyAsync(dev, buf.data(), bytes, cudaMemcpyHostToDevice, b->stream)
                              : cudaSuccess;
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        return e == cudaSuccess ? PIC_OK : cuda_fail(b, e, "restore");
    };
    pic_status st = PIC_OK;
    for (int c = 0; c < 5 && st == PIC_OK; ++c) st = get(r.dev.F[0][c], r.glen * 4);
    std::vector<float> jsaved(3 * r.glen);
    if (std::fread(jsaved.data(), 4, jsaved.size(), f) != jsaved.size())
        return fail(b, PIC_ERR_INVALID_ARG, "checkpoint file is truncated");
    for (int s = 0; s < 2 && st == PIC_OK; ++s) {
        if (!h.loaded[s]) continue;
        if ((st = alloc_species(b, r, s, h.n[s])) != PIC_OK) break;
        const DevSpecies& d = r.dev.sp[s][b->cur];
        const size_t by = static_cast<size_t>(h.n[s]) * 4;
        for (void* a : {static_cast<void*>(d.cell), static_cast<void*>(d.off), static_cast<void*>(d.px),
                        static_cast<void*>(d.py), static_cast<void*>(d.pz), static_cast<void*>(d.id)})
            if (st == PIC_OK) st = get(a, by);
        r.sp[s].loaded = true;
        r.sp[s].w = h.w[s];
        r.sp[s].q = h.q[s];
        r.sp[s].m = h.m[s];
    }
    if (st != PIC_OK) return st;
    PIC_CK(b, cudaMemcpy(r.dev.tally, h.tally, sizeof(h.tally), cudaMemcpyHostToDevice));
    if (h.laser_on) {
        r.laser.on = 1;
        r.laser.pol = h.pol;
        r.laser.env = h.env;
        r.laser.a0 = h.a0;
        r.laser.tau = h.tau;
        r.laser.rise = h.rise;
        r.laser_set = true;
    }
    r.fields_set = true;
    r.t_offset = h.steps;
    // the saved current goes into the accumulator set a run reads back before
    // its first step (1), in the fixed-point scale the run will step with
    finalize_run_params(b, r);
    std::vector<long long> acc(r.glen);
    for (int c = 0; c < 3; ++c) {
        for (size_t i = 0; i < r.glen; ++i)
            acc[i] = std::llround(std::ldexp(static_cast<double>(jsaved[c * r.glen + i]), r.fp_bits));
        PIC_CK(b, cudaMemcpy(r.dev.J[1][c], acc.data(), sizeof(long long) * r.glen, cudaMemcpyHostToDevice));
    }
    return PIC_OK;
}

void fill_stats(Batch* b, pic_stats_t* out) {
    std::memset(out, 0, sizeof(*out));
    out->steps = b->gstep;
    out->kernel_launches = b->launches;
    out->push_launches = b->push_launches;
    out->sort_count = b->sorts;
    out->push_ms = b->push_ms;
    out->field_ms = b->field_ms;
    out->sort_ms = b->sort_ms;
    out->timed_push_launches = b->timed_push;
    out->graph_launches = b->graph_launches;
    out->steps_since_sort = b->since_sort;
    out->device_bytes = static_cast<int64_t>(b->bytes);
    int64_t act = 0;
    int fp = 0;
    for (auto& r : b->runs) {
        if (!r.used || r.finished) continue;
        for (int s = 0; s < 2; ++s) act += r.sp[s].loaded ? r.sp[s].n : 0;
        if (r.started) fp = r.fp_bits;
    }
    out->active_particles = act;
    out->fp_bits = fp;
    int32_t cnt = 0;
    if (b->units.count && cudaMemcpy(&cnt, b->units.count, sizeof(int32_t), cudaMemcpyDeviceToHost) == cudaSuccess)
        out->n_units = cnt;
}

pic_status set_timing(Batch* b, int on) {
    DeviceGuard g(b->device);
    cudaStreamSynchronize(b->stream);
    collect_timing(b);
    read_all_graph_timing(b);
    b->timing = on != 0;
    if (b->timing) {
        b->push_ms = b->field_ms = b->sort_ms = 0.0;
        b->timed_push = 0;
    }
    return PIC_OK;
}

}  // namespace
}  // namespace picrr

using namespace picrr;

// A single-run handle: a batch of one.
struct pic_sim {
    Batch* b = nullptr;
};

struct pic_batch {
    Batch* b = nullptr;
};

extern "C" {

// ---------------------------------------------------------------------------
// single run
// ---------------------------------------------------------------------------

pic_status pic_create(const pic_config* cfg, pic_sim** out) {
    if (!out) return fail(nullptr, PIC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!cfg) return fail(nullptr, PIC_ERR_INVALID_ARG, "cfg is NULL");
    pic_status st = validate_common(cfg);
    if (st != PIC_OK) return st;
    const double ncell = cfg->length_lambda * cfg->cells_per_lambda;
    if (!(cfg->length_lambda > 0.0) || !(ncell >= 16.0 && ncell <= 1.0e9))
        return fail(nullptr, PIC_ERR_INVALID_ARG, "Nx must be in [16, 1e9]");
    const int Nx = static_cast<int>(std::llround(ncell));
    const int is = cfg->source_node ? cfg->source_node : 8;
    if (is < 2 || is > Nx - 4) return fail(nullptr, PIC_ERR_INVALID_ARG, "source_node must be in [2, Nx-4]");
    Batch* b = nullptr;
    if ((st = batch_create(cfg, 1, &b)) != PIC_OK) return st;
    DeviceGuard g(b->device);
    int id = -1;
    st = run_open(b, cfg->length_lambda, is, cfg->rr_on, cfg->seed, &id);
    if (st == PIC_OK && cudaStreamSynchronize(b->stream) != cudaSuccess) st = cuda_fail(b, cudaGetLastError(), "create");
    if (st != PIC_OK) {
        g_null_error = b->err;
        batch_destroy(b);
        return st;
    }
    pic_sim* s = new pic_sim();
    s->b = b;
    *out = s;
    return PIC_OK;
}

pic_status pic_set_stream(pic_sim* s, void* stream) {
    if (!s) return PIC_ERR_INVALID_ARG;
    DeviceGuard g(s->b->device);
    cudaStreamSynchronize(s->b->stream);
    s->b->stream = stream ? static_cast<cudaStream_t>(stream) : s->b->own_stream;
    return PIC_OK;
}

pic_status pic_load_foil(pic_sim* s, double x0_lambda, double thickness_lambda, double ne_over_nc, int ion_Z,
                         double ion_A, int ppc) {
    if (!s) return PIC_ERR_INVALID_ARG;
    DeviceGuard g(s->b->device);
    pic_status st = run_load_foil(s->b, 0, x0_lambda, thickness_lambda, ne_over_nc, ion_Z, ion_A, ppc);
    if (st != PIC_OK) return st;
    cudaError_t e = cudaStreamSynchronize(s->b->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? PIC_OK : cuda_fail(s->b, e, "foil loader");
}

pic_status pic_load_particles(pic_sim* s, int species, int64_t n, const int32_t* cell, const double* off,
                              const double* px, const double* py, const double* pz, double weight, double charge,
                              double mass) {
    if (!s) return PIC_ERR_INVALID_ARG;
    Batch* b = s->b;
    RunHost& r = b->runs[0];
    pic_status st = check_species_args(b, r, species, n, weight, charge, mass);
    if (st != PIC_OK) return st;
    if (n > 0 && (!cell || !off || !px || !py || !pz)) return fail(b, PIC_ERR_INVALID_ARG, "NULL array");
    std::vector<float> o(static_cast<size_t>(n)), x(static_cast<size_t>(n)), y(static_cast<size_t>(n)),
        z(static_cast<size_t>(n));
    for (int64_t i = 0; i < n; ++i) {
        if (!std::isfinite(px[i]) || !std::isfinite(py[i]) || !std::isfinite(pz[i]) || !std::isfinite(off[i]))
            return fail(b, PIC_ERR_INVALID_ARG, "non-finite input");
        o[i] = static_cast<float>(off[i]);
        x[i] = static_cast<float>(px[i]);
        y[i] = static_cast<float>(py[i]);
        z[i] = static_cast<float>(pz[i]);
    }
    DeviceGuard g(b->device);
    return run_load_particles_f32(b, 0, species, n, cell, o.data(), x.data(), y.data(), z.data(), weight, charge,
                                  mass);
}

pic_status pic_load_particles_f32(pic_sim* s, int species, int64_t n, const int32_t* cell, const float* off,
                                  const float* px, const float* py, const float* pz, double weight, double charge,
                                  double mass) {
    if (!s) return PIC_ERR_INVALID_ARG;
    DeviceGuard g(s->b->device);
    return run_load_particles_f32(s->b, 0, species, n, cell, off, px, py, pz, weight, charge, mass);
}

pic_status pic_set_fields(pic_sim* s, const double* Ex, const double* Ey, const double* Ez, const double* By,
                          const double* Bz) {
    if (!s) return PIC_ERR_INVALID_ARG;
    DeviceGuard g(s->b->device);
    const double* src[5] = {Ex, Ey, Ez, By, Bz};
    return run_set_fields(s->b, 0, src);
}

pic_status pic_inject_laser(pic_sim* s, double a0, int polarization, int envelope, double duration_periods,
                            double rise_periods) {
    if (!s) return PIC_ERR_INVALID_ARG;
    return run_inject_laser(s->b, 0, a0, polarization, envelope, duration_periods, rise_periods);
}

pic_status pic_step_n(pic_sim* s, int64_t n, int64_t* steps_done) {
    if (steps_done) *steps_done = 0;
    if (!s) return PIC_ERR_INVALID_ARG;
    if (n < 0) return fail(s->b, PIC_ERR_INVALID_ARG, "n must be >= 0");
    DeviceGuard g(s->b->device);
    return batch_step(s->b, n, steps_done);
}

pic_status pic_energy(pic_sim* s, double out[6]) {
    if (!s) return PIC_ERR_INVALID_ARG;
    if (!out) return fail(s->b, PIC_ERR_INVALID_ARG, "out is NULL");
    DeviceGuard g(s->b->device);
    return run_energy(s->b, 0, out);
}

pic_status pic_spectra(pic_sim* s, int species, int nbins, double e_min, double e_max, double* counts,
                       double* radiated) {
    if (!s) return PIC_ERR_INVALID_ARG;
    DeviceGuard g(s->b->device);
    return run_spectra(s->b, 0, species, nbins, e_min, e_max, counts, radiated);
}

pic_status pic_read_particles(pic_sim* s, int species, int64_t cap, double* x, double* px, double* py, double* pz,
                              int32_t* flag, int64_t* n) {
    if (!s) return PIC_ERR_INVALID_ARG;
    DeviceGuard g(s->b->device);
    return run_read_particles(s->b, 0, species, cap, x, px, py, pz, flag, n);
}

pic_status pic_snapshot(pic_sim* s, int species, double chi_flag, int64_t cap, double* x, double* px, double* pperp,
                        double* d, double* chi, double* summary, int64_t* n) {
    if (!s) return PIC_ERR_INVALID_ARG;
    DeviceGuard g(s->b->device);
    return run_snapshot(s->b, 0, species, chi_flag, cap, x, px, pperp, d, chi, summary, n);
}

pic_status pic_read_fields(pic_sim* s, int comp, int64_t cap, double* out, int64_t* n) {
    if (!s) return PIC_ERR_INVALID_ARG;
    DeviceGuard g(s->b->device);
    return run_read_fields(s->b, 0, comp, cap, out, n);
}

pic_status pic_tune_shapes(pic_sim* s, int64_t steps_per_candidate, int* unit_particles, int* sort_interval,
                           int* particles_per_thread, double* ms_per_step) {
    if (!s) return PIC_ERR_INVALID_ARG;
    DeviceGuard g(s->b->device);
    return tune_shapes(s->b, steps_per_candidate, unit_particles, sort_interval, particles_per_thread, ms_per_step);
}

pic_status pic_set_shapes(pic_sim* s, int unit_particles, int sort_interval, int particles_per_thread) {
    if (!s) return PIC_ERR_INVALID_ARG;
    DeviceGuard g(s->b->device);
    return set_shapes(s->b, unit_particles, sort_interval, particles_per_thread);
}

pic_status pic_stats(pic_sim* s, pic_stats_t* out) {
    if (!s || !out) return PIC_ERR_INVALID_ARG;
    DeviceGuard g(s->b->device);
    cudaStreamSynchronize(s->b->stream);
    fill_stats(s->b, out);
    return PIC_OK;
}

pic_status pic_set_timing(pic_sim* s, int on) {
    if (!s) return PIC_ERR_INVALID_ARG;
    return set_timing(s->b, on);
}

pic_status pic_set_rr(pic_sim* s, int rr_on) {
    if (!s) return PIC_ERR_INVALID_ARG;
    if (rr_on != 0 && rr_on != 1) return fail(s->b, PIC_ERR_INVALID_ARG, "rr_on must be 0 or 1");
    RunHost& r = s->b->runs[0];
    r.rr = rr_on;
    r.dev.rr = rr_on;  // the kernels read the run table at run time: no graph recapture
    s->b->table_dirty = true;
    return PIC_OK;
}

const char* pic_last_error(const pic_sim* s) { return s ? s->b->err.c_str() : g_null_error.c_str(); }

pic_status pic_get_config(const pic_sim* s, pic_config* out) {
    if (!s || !out) return PIC_ERR_INVALID_ARG;
    const Batch* b = s->b;
    const RunHost& r = b->runs[0];
    *out = b->cfg;
    out->length_lambda = r.length_lambda;
    out->rr_on = r.rr;
    out->seed = r.seed;
    out->source_node = r.is;
    out->sort_interval = b->sort_interval;
    return PIC_OK;
}

pic_status pic_save(pic_sim* s, const char* path) {
    if (!s) return PIC_ERR_INVALID_ARG;
    if (!path) return fail(s->b, PIC_ERR_INVALID_ARG, "path is NULL");
    DeviceGuard g(s->b->device);
    return run_save(s->b, 0, path);
}

pic_status pic_restore(const char* path, int device, int sort_interval, pic_sim** out) {
    if (!out) return fail(nullptr, PIC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!path) return fail(nullptr, PIC_ERR_INVALID_ARG, "path is NULL");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(nullptr, PIC_ERR_INVALID_ARG, std::string("cannot open ") + path);
    CkHeader h{};
    if (std::fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, kMagic, 8) != 0 || h.version != 1 ||
        h.n[0] < 0 || h.n[1] < 0 || h.n[0] > 2147483647LL - 64 || h.n[1] > 2147483647LL - 64) {
        std::fclose(f);
        return fail(nullptr, PIC_ERR_INVALID_ARG, "not a picrr checkpoint (or another version)");
    }
    pic_config cfg{};
    cfg.length_lambda = h.length_lambda;
    cfg.cells_per_lambda = h.cells_per_lambda;
    cfg.cfl = h.cfl;
    cfg.lambda_um = h.lambda_um;
    cfg.rr_on = h.rr;
    cfg.sort_interval = sort_interval;
    cfg.seed = h.seed;
    cfg.device = device;
    cfg.source_node = h.source_node;
    pic_sim* s = nullptr;
    pic_status st = pic_create(&cfg, &s);
    if (st != PIC_OK) {
        std::fclose(f);
        return st;
    }
    if (s->b->runs[0].Nx != h.nx || static_cast<int64_t>(s->b->runs[0].glen) != h.glen) {
        std::fclose(f);
        pic_destroy(s);
        return fail(nullptr, PIC_ERR_INVALID_ARG, "checkpoint grid does not match its configuration");
    }
    {
        DeviceGuard g(s->b->device);
        st = run_restore(s->b, 0, f, h);
    }
    std::fclose(f);
    if (st != PIC_OK) {
        g_null_error = s->b->err;
        pic_destroy(s);
        return st;
    }
    *out = s;
    return PIC_OK;
}

pic_status pic_selftest_wait_timeout(int device, double* seconds) {
    if (seconds) *seconds = 0.0;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, PIC_ERR_INVALID_ARG, "bad device");
    }
    int* d_status = nullptr;
    int h = 0;
    const auto t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaMalloc(&d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(d_status, 0, sizeof(int));
    if (e == cudaSuccess) {
        launch_wait_selftest(d_status, nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (d_status) cudaFree(d_status);
    if (seconds) *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "wait self-test");
    if (h & ST_TIMEOUT) return fail(nullptr, PIC_ERR_TIMEOUT, "bounded device wait gave up (expected)");
    return PIC_OK;
}

pic_status pic_destroy(pic_sim* s) {
    if (!s) return PIC_OK;
    batch_destroy(s->b);
    delete s;
    return PIC_OK;
}

// ---------------------------------------------------------------------------
// batch of runs
// ---------------------------------------------------------------------------

pic_status pic_batch_create(const pic_config* common, int max_runs, pic_batch** out) {
    if (!out) return fail(nullptr, PIC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    Batch* b = nullptr;
    pic_status st = batch_create(common, max_runs, &b);
    if (st != PIC_OK) return st;
    pic_batch* h = new pic_batch();
    h->b = b;
    *out = h;
    return PIC_OK;
}

pic_status pic_batch_set_stream(pic_batch* h, void* stream) {
    if (!h) return PIC_ERR_INVALID_ARG;
    DeviceGuard g(h->b->device);
    cudaStreamSynchronize(h->b->stream);
    h->b->stream = stream ? static_cast<cudaStream_t>(stream) : h->b->own_stream;
    return PIC_OK;
}

pic_status pic_batch_add_run(pic_batch* h, const pic_run_desc* d, int* run_id) {
    if (!h) return PIC_ERR_INVALID_ARG;
    Batch* b = h->b;
    if (!d || !run_id) return fail(b, PIC_ERR_INVALID_ARG, "desc and run_id must not be NULL");
    *run_id = -1;
    if (d->steps < 1) return fail(b, PIC_ERR_INVALID_ARG, "steps must be >= 1");
    DeviceGuard g(b->device);
    int id = -1;
    pic_status st = run_open(b, d->length_lambda, d->source_node, d->rr_on, d->seed, &id);
    if (st != PIC_OK) return st;
    if ((st = run_load_foil(b, id, d->foil_x0_lambda, d->foil_thickness_lambda, d->ne_over_nc, d->ion_Z, d->ion_A,
                            d->ppc)) != PIC_OK ||
        (st = run_inject_laser(b, id, d->a0, d->polarization, d->envelope, d->duration_periods,
                               d->rise_periods)) != PIC_OK) {
        run_release(b, id);
        return st;
    }
    b->runs[id].steps_target = d->steps;
    *run_id = id;
    return PIC_OK;
}

pic_status pic_batch_run_footprint(const pic_batch* h, const pic_run_desc* d, size_t* bytes) {
    // reads only the batch's configuration and reports errors through the
    // calling thread's handle-less message, so it may run beside the batch's owner
    if (!h) return PIC_ERR_INVALID_ARG;
    if (!d || !bytes) return fail(nullptr, PIC_ERR_INVALID_ARG, "desc and bytes must not be NULL");
    const double cpl = h->b->cfg.cells_per_lambda, ncell = d->length_lambda * cpl;
    if (!(d->length_lambda > 0.0) || !(ncell >= 16.0 && ncell <= 1.0e9) || d->ppc < 1 ||
        !(d->foil_thickness_lambda > 0.0) || !(d->foil_thickness_lambda * cpl < 1.0e9))
        return fail(nullptr, PIC_ERR_INVALID_ARG, "need 16 <= cells <= 1e9, ppc >= 1, thickness > 0");
    const int64_t n = std::llround(d->foil_thickness_lambda * cpl) * static_cast<int64_t>(d->ppc);
    *bytes = run_footprint(h->b, d->length_lambda, n);
    return PIC_OK;
}

pic_status pic_shard_runs(const pic_config* common, const pic_run_desc* runs, int n_runs, int n_ranks,
                          int in_order, size_t budget_per_rank, int* rank_of_run, double* work_per_rank) {
    if (!common || (n_runs > 0 && (!runs || !rank_of_run)) || n_runs < 0 || n_ranks < 1)
        return fail(nullptr, PIC_ERR_INVALID_ARG, "need a config, n_runs >= 0 runs and ranks, n_ranks >= 1");
    const double cpl = common->cells_per_lambda;
    if (!(cpl > 0.0)) return fail(nullptr, PIC_ERR_INVALID_ARG, "cells_per_lambda must be > 0");
    std::vector<double> work(static_cast<size_t>(n_runs));
    std::vector<size_t> foot(static_cast<size_t>(n_runs));
    for (int i = 0; i < n_runs; ++i) {
        const pic_run_desc& d = runs[i];
        const double ncell = d.length_lambda * cpl;
        if (!(d.length_lambda > 0.0) || !(ncell >= 16.0 && ncell <= 1.0e9) || d.ppc < 1 ||
            !(d.foil_thickness_lambda > 0.0) || !(d.foil_thickness_lambda * cpl < 1.0e9) || d.steps < 1)
            return fail(nullptr, PIC_ERR_INVALID_ARG,
                        "run " + std::to_string(i) + ": need 16 <= cells <= 1e9, ppc >= 1, thickness > 0, steps >= 1");
        const int64_t n = std::llround(d.foil_thickness_lambda * cpl) * static_cast<int64_t>(d.ppc);
        work[i] = 2.0 * static_cast<double>(n) * static_cast<double>(d.steps);
        foot[i] = run_footprint_cpl(cpl, d.length_lambda, n);
    }
    std::vector<int> order(static_cast<size_t>(n_runs));
    for (int i = 0; i < n_runs; ++i) order[i] = i;
    if (!in_order)  // largest work first; equal work keeps the index order
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
    std::vector<double> load(static_cast<size_t>(n_ranks), 0.0);
    std::vector<size_t> mem(static_cast<size_t>(n_ranks), 0);
    std::vector<int> out(static_cast<size_t>(n_runs), -1);
    for (int i : order) {
        int best = -1;
        for (int r = 0; r < n_ranks; ++r) {
            if (budget_per_rank && mem[r] + foot[i] > budget_per_rank) continue;
            if (best < 0 || load[r] < load[best]) best = r;  // ties: the lowest rank
        }
        if (best < 0)
            return fail(nullptr, PIC_ERR_OOM, "run " + std::to_string(i) + " fits no rank's memory budget");
        out[i] = best;
        load[best] += work[i];
        mem[best] += foot[i];
    }
    for (int i = 0; i < n_runs; ++i) rank_of_run[i] = out[i];
    if (work_per_rank)
        for (int r = 0; r < n_ranks; ++r) work_per_rank[r] = load[r];
    return PIC_OK;
}

pic_status pic_batch_step(pic_batch* h, int64_t n, int64_t* steps_done) {
    if (steps_done) *steps_done = 0;
    if (!h) return PIC_ERR_INVALID_ARG;
    if (n < 0) return fail(h->b, PIC_ERR_INVALID_ARG, "n must be >= 0");
    DeviceGuard g(h->b->device);
    return batch_step(h->b, n, steps_done);
}

static pic_status check_run(pic_batch* h, int run) {
    if (!h) return PIC_ERR_INVALID_ARG;
    if (run < 0 || run >= h->b->max_runs || !h->b->runs[run].used)
        return fail(h->b, PIC_ERR_INVALID_ARG, "no such run");
    return PIC_OK;
}

pic_status pic_batch_run_status(pic_batch* h, int run, int64_t* steps_done, int* finished) {
    pic_status st = check_run(h, run);
    if (st != PIC_OK) return st;
    const RunHost& r = h->b->runs[run];
    if (steps_done) *steps_done = r.steps_done;
    if (finished) *finished = r.finished ? 1 : 0;
    return PIC_OK;
}

pic_status pic_batch_energy(pic_batch* h, int run, double out[6]) {
    pic_status st = check_run(h, run);
    if (st != PIC_OK) return st;
    if (!out) return fail(h->b, PIC_ERR_INVALID_ARG, "out is NULL");
    DeviceGuard g(h->b->device);
    return run_energy(h->b, run, out);
}

pic_status pic_batch_spectra(pic_batch* h, int run, int species, int nbins, double e_min, double e_max,
                             double* counts, double* radiated) {
    pic_status st = check_run(h, run);
    if (st != PIC_OK) return st;
    DeviceGuard g(h->b->device);
    return run_spectra(h->b, run, species, nbins, e_min, e_max, counts, radiated);
}

pic_status pic_batch_read_particles(pic_batch* h, int run, int species, int64_t cap, double* x, double* px,
                                    double* py, double* pz, int32_t* flag, int64_t* n) {
    pic_status st = check_run(h, run);
    if (st != PIC_OK) return st;
    DeviceGuard g(h->b->device);
    return run_read_particles(h->b, run, species, cap, x, px, py, pz, flag, n);
}

pic_status pic_batch_snapshot(pic_batch* h, int run, int species, double chi_flag, int64_t cap, double* x, double* px,
                              double* pperp, double* d, double* chi, double* summary, int64_t* n) {
    pic_status st = check_run(h, run);
    if (st != PIC_OK) return st;
    DeviceGuard g(h->b->device);
    return run_snapshot(h->b, run, species, chi_flag, cap, x, px, pperp, d, chi, summary, n);
}

pic_status pic_batch_read_fields(pic_batch* h, int run, int comp, int64_t cap, double* out, int64_t* n) {
    pic_status st = check_run(h, run);
    if (st != PIC_OK) return st;
    DeviceGuard g(h->b->device);
    return run_read_fields(h->b, run, comp, cap, out, n);
}

pic_status pic_batch_stop_run(pic_batch* h, int run) {
    pic_status st = check_run(h, run);
    if (st != PIC_OK) return st;
    Batch* b = h->b;
    RunHost& r = b->runs[run];
    if (!r.active) return PIC_OK;  // not stepping (pending, finished or stopped)
    DeviceGuard g(b->device);
    if (b->since_sort > 0) rad_flush(b);  // the run takes its radiated energy with it
    deactivate(b, run);
    if ((st = upload_table(b)) != PIC_OK) return st;
    return upload_blocks(b);
}

pic_status pic_batch_release_run(pic_batch* h, int run) {
    pic_status st = check_run(h, run);
    if (st != PIC_OK) return st;
    Batch* b = h->b;
    if (b->runs[run].active) return fail(b, PIC_ERR_STATE, "run is still stepping");
    DeviceGuard g(b->device);
    run_release(b, run);
    return upload_table(b);
}

pic_status pic_batch_tune_shapes(pic_batch* h, int64_t steps_per_candidate, int* unit_particles, int* sort_interval,
                                 int* particles_per_thread, double* ms_per_step) {
    if (!h) return PIC_ERR_INVALID_ARG;
    DeviceGuard g(h->b->device);
    return tune_shapes(h->b, steps_per_candidate, unit_particles, sort_interval, particles_per_thread, ms_per_step);
}

pic_status pic_batch_set_shapes(pic_batch* h, int unit_particles, int sort_interval, int particles_per_thread) {
    if (!h) return PIC_ERR_INVALID_ARG;
    DeviceGuard g(h->b->device);
    return set_shapes(h->b, unit_particles, sort_interval, particles_per_thread);
}

pic_status pic_batch_stats(pic_batch* h, pic_stats_t* out) {
    if (!h || !out) return PIC_ERR_INVALID_ARG;
    DeviceGuard g(h->b->device);
    cudaStreamSynchronize(h->b->stream);
    fill_stats(h->b, out);
    return PIC_OK;
}

pic_status pic_batch_set_timing(pic_batch* h, int on) {
    if (!h) return PIC_ERR_INVALID_ARG;
    return set_timing(h->b, on);
}

const char* pic_batch_last_error(const pic_batch* h) { return h ? h->b->err.c_str() : g_null_error.c_str(); }

pic_status pic_batch_destroy(pic_batch* h) {
    if (!h) return PIC_OK;
    batch_destroy(h->b);
    delete h;
    return PIC_OK;
}

}  // extern "C"
