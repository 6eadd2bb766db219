// Serving loop of the picrr C ABI: a worker thread that owns one batch,
// admits queued run requests (in arrival order, or shortest work first) as
// slots, the device-memory budget and an optional cap on resident particles
// allow, steps the batch in chunks (requests join between chunks while
// the others keep stepping), and turns every finished run into its spectra
// and energy read-out before freeing it.  Built only on the public
// pic_batch_* entry points; host code only.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "picrr.h"

namespace {

using Clock = std::chrono::steady_clock;

thread_local std::string t_err;  // last failed server call of this thread

pic_status sfail(pic_status st, const std::string& msg) {
    t_err = msg;
    return st;
}

enum ReqState { QUEUED, RUNNING, DONE, FAILED };

struct Request {
    int64_t ticket = 0;
    pic_run_desc desc{};
    int nbins = 0;
    double ion_max = 0.0, el_max = 0.0;
    size_t footprint = 0;
    int64_t particles = 0;
    double work = 0.0;  // particles x steps
    Clock::time_point submitted;
    ReqState state = QUEUED;
    bool cancel = false;  // asked to stop while running
    int run = -1;
    int64_t steps_seen = 0;
    std::vector<double> ion, el;
    double energy[6] = {0, 0, 0, 0, 0, 0};
    double latency = 0.0;
    pic_status status = PIC_OK;
    std::string err;
};

}  // namespace

struct pic_server {
    pic_batch* batch = nullptr;
    int max_runs = 0;
    int64_t chunk = 0;
    size_t budget = 0;
    double cells_per_lambda = 0.0;

    std::mutex m;
    std::condition_variable cv_work, cv_done;
    std::deque<int64_t> queue;
    std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
    int64_t next_ticket = 1;
    bool stop = false;
    pic_status fatal = PIC_OK;
    int policy = PIC_SERVE_FIFO;
    int64_t max_resident = 0;  // particles resident at once (0: no cap)
    int64_t resident = 0;
    std::string fatal_msg;
    pic_server_stats_t st{};
    std::thread worker;

    void run();
    void finish_run(Request* r);
    void fail_all(pic_status s, const std::string& msg);
};

void pic_server::fail_all(pic_status s, const std::string& msg) {
    std::lock_guard<std::mutex> lk(m);
    fatal = s;
    fatal_msg = msg;
    for (auto& kv : reqs) {
        Request* r = kv.second.get();
        if (r->state == QUEUED || r->state == RUNNING) {
            r->state = FAILED;
            r->status = s;
            r->err = msg;
            st.failed++;
        }
    }
    queue.clear();
    st.queued = st.running = 0;
    cv_done.notify_all();
}

// Read-outs of a finished run, then free it.
void pic_server::finish_run(Request* r) {
    std::vector<double> ion(static_cast<size_t>(r->nbins)), el(static_cast<size_t>(r->nbins));
    double e[6];
    pic_status s = pic_batch_spectra(batch, r->run, PIC_ION, r->nbins, 0.0, r->ion_max, ion.data(), nullptr);
    if (s == PIC_OK) s = pic_batch_spectra(batch, r->run, PIC_ELECTRON, r->nbins, 0.0, r->el_max, el.data(), nullptr);
    if (s == PIC_OK) s = pic_batch_energy(batch, r->run, e);
    const std::string msg = s == PIC_OK ? std::string() : pic_batch_last_error(batch);
    pic_batch_release_run(batch, r->run);
    const double lat = std::chrono::duration<double>(Clock::now() - r->submitted).count();
    std::lock_guard<std::mutex> lk(m);
    r->run = -1;
    resident -= r->particles;
    st.running--;
    if (s == PIC_OK) {
        r->ion.swap(ion);
        r->el.swap(el);
        for (int k = 0; k < 6; ++k) r->energy[k] = e[k];
        r->latency = lat;
        r->state = DONE;
        st.completed++;
    } else {
        r->state = FAILED;
        r->status = s;
        r->err = msg;
        st.failed++;
    }
    cv_done.notify_all();
}

void pic_server::run() {
    std::vector<Request*> running;
    for (;;) {
        std::vector<Request*> admit;
        if (running.empty()) {
            std::unique_lock<std::mutex> lk(m);
            cv_work.wait(lk, [&] { return stop || !queue.empty(); });
        }
        pic_stats_t bs{};
        pic_batch_stats(batch, &bs);  // the batch is only touched by this thread
        {
            std::unique_lock<std::mutex> lk(m);
            if (stop) return;
            // admission: the next request by the policy waits for room
            size_t used = static_cast<size_t>(bs.device_bytes);
            int free_slots = max_runs - static_cast<int>(running.size());
            int64_t res = resident;
            while (!queue.empty() && free_slots > 0) {
                size_t pick = 0;
                if (policy == PIC_SERVE_SHORTEST_FIRST)
                    for (size_t q = 1; q < queue.size(); ++q)
                        if (reqs[queue[q]]->work < reqs[queue[pick]]->work) pick = q;
                Request* r = reqs[queue[pick]].get();
                // (with nothing resident, the request is admitted: it fits the budget alone)
                const bool alone = running.empty() && admit.empty();
                if (budget && used + r->footprint > budget && !alone) break;
                if (max_resident && res + r->particles > max_resident && !alone) break;
                queue.erase(queue.begin() + static_cast<long>(pick));
                admit.push_back(r);
                used += r->footprint;
                res += r->particles;
                free_slots--;
            }
            st.queued = static_cast<int64_t>(queue.size());
        }
        for (size_t i = 0; i < admit.size(); ++i) {
            Request* r = admit[i];
            int id = -1;
            const pic_status s = pic_batch_add_run(batch, &r->desc, &id);
            std::lock_guard<std::mutex> lk(m);
            if (s == PIC_OK) {
                r->run = id;
                r->state = RUNNING;
                running.push_back(r);
                resident += r->particles;
                st.admitted++;
                st.running++;
            } else if (s == PIC_ERR_OOM && !running.empty()) {
                // no room after all: back to the head of the queue, in order
                for (size_t j = admit.size(); j-- > i;) queue.push_front(admit[j]->ticket);
                st.queued = static_cast<int64_t>(queue.size());
                break;
            } else {
                r->state = FAILED;
                r->status = s;
                r->err = pic_batch_last_error(batch);
                st.failed++;
                cv_done.notify_all();
            }
        }
        if (running.empty()) continue;
        {
            pic_stats_t bs{};
            pic_batch_stats(batch, &bs);
            std::lock_guard<std::mutex> lk(m);
            if (bs.device_bytes > st.peak_device_bytes) st.peak_device_bytes = bs.device_bytes;
            st.device_bytes = bs.device_bytes;
        }
        const auto t0 = Clock::now();
        int64_t done = 0;
        const pic_status s = pic_batch_step(batch, chunk, &done);
        const double dt = std::chrono::duration<double>(Clock::now() - t0).count();
        if (s != PIC_OK) {
            fail_all(s, std::string("batch step: ") + pic_batch_last_error(batch));
            return;
        }
        int64_t ps = 0;
        std::vector<Request*> still;
        std::vector<Request*> ended;
        for (Request* r : running) {
            int64_t sd = 0;
            int fin = 0;
            pic_batch_run_status(batch, r->run, &sd, &fin);
            ps += (sd - r->steps_seen) * r->particles;
            r->steps_seen = sd;
            (fin ? ended : still).push_back(r);
        }
        {
            std::lock_guard<std::mutex> lk(m);
            st.batch_steps += done;
            st.particle_steps += ps;
            st.busy_s += dt;
        }
        for (Request* r : ended) finish_run(r);
        running.swap(still);
        // cancelled requests leave the batch between chunks
        std::vector<Request*> keep;
        for (Request* r : running) {
            bool c;
            {
                std::lock_guard<std::mutex> lk(m);
                c = r->cancel;
            }
            if (!c) {
                keep.push_back(r);
                continue;
            }
            pic_batch_stop_run(batch, r->run);
            pic_batch_release_run(batch, r->run);
            std::lock_guard<std::mutex> lk(m);
            r->run = -1;
            resident -= r->particles;
            st.running--;
            r->state = FAILED;
            r->status = PIC_ERR_STATE;
            r->err = "cancelled";
            st.failed++;
            cv_done.notify_all();
        }
        running.swap(keep);
    }
}

extern "C" {

pic_status pic_server_create(const pic_config* common, int max_runs, int64_t chunk_steps, pic_server** out) {
    if (!out) return sfail(PIC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!common) return sfail(PIC_ERR_INVALID_ARG, "common is NULL");
    if (chunk_steps < 1) return sfail(PIC_ERR_INVALID_ARG, "chunk_steps must be >= 1");
    pic_batch* b = nullptr;
    pic_status s = pic_batch_create(common, max_runs, &b);
    if (s != PIC_OK) return sfail(s, pic_batch_last_error(nullptr));
    auto* v = new pic_server();
    v->batch = b;
    v->max_runs = max_runs;
    const int64_t si = common->sort_interval ? common->sort_interval : 8;
    // chunks end on sort boundaries, so runs join without an early sort of the others
    v->chunk = (chunk_steps + si - 1) / si * si;
    v->budget = common->hbm_budget_bytes;
    v->cells_per_lambda = common->cells_per_lambda;
    v->worker = std::thread([v] { v->run(); });
    *out = v;
    return PIC_OK;
}

pic_status pic_server_submit(pic_server* v, const pic_run_desc* d, int nbins, double ion_e_max_MeV,
                             double el_e_max_MeV, int64_t* ticket) {
    if (!v) return sfail(PIC_ERR_INVALID_ARG, "server is NULL");
    if (!d || !ticket) return sfail(PIC_ERR_INVALID_ARG, "desc and ticket must not be NULL");
    *ticket = 0;
    if (nbins < 1 || nbins > (1 << 24) || !(ion_e_max_MeV > 0.0) || !(el_e_max_MeV > 0.0))
        return sfail(PIC_ERR_INVALID_ARG, "need 1 <= nbins <= 2^24 and positive energy ranges");
    size_t fp = 0;
    pic_status s = pic_batch_run_footprint(v->batch, d, &fp);  // reads only the batch's configuration
    if (s != PIC_OK) return sfail(s, "invalid run description: " + std::string(pic_batch_last_error(nullptr)));
    if (v->budget && fp > v->budget)
        return sfail(PIC_ERR_OOM, "run needs " + std::to_string(fp) + " bytes, over the budget of " +
                                      std::to_string(v->budget));
    auto r = std::make_unique<Request>();
    r->desc = *d;
    r->nbins = nbins;
    r->ion_max = ion_e_max_MeV;
    r->el_max = el_e_max_MeV;
    r->footprint = fp;
    r->particles = 2 * static_cast<int64_t>(std::llround(d->foil_thickness_lambda * v->cells_per_lambda)) * d->ppc;
    r->work = static_cast<double>(r->particles) * static_cast<double>(d->steps);
    r->submitted = Clock::now();
    std::lock_guard<std::mutex> lk(v->m);
    if (v->fatal != PIC_OK) return sfail(v->fatal, "server stopped: " + v->fatal_msg);
    r->ticket = v->next_ticket++;
    *ticket = r->ticket;
    v->queue.push_back(r->ticket);
    v->reqs.emplace(r->ticket, std::move(r));
    v->st.submitted++;
    v->st.queued = static_cast<int64_t>(v->queue.size());
    v->cv_work.notify_one();
    return PIC_OK;
}

pic_status pic_server_result(pic_server* v, int64_t ticket, double wait_s, double* ion_counts, double* el_counts,
                             double* energy, double* latency_s) {
    if (!v) return sfail(PIC_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(v->m);
    auto it = v->reqs.find(ticket);
    if (it == v->reqs.end()) return sfail(PIC_ERR_INVALID_ARG, "unknown ticket");
    Request* r = it->second.get();
    auto ready = [&] { return r->state == DONE || r->state == FAILED; };
    if (!ready() && wait_s > 0.0)
        v->cv_done.wait_for(lk, std::chrono::duration<double>(wait_s), ready);
    if (!ready()) return sfail(PIC_ERR_TIMEOUT, "request not finished");
    if (r->state == FAILED) {
        const pic_status s = r->status;
        const std::string msg = r->err;
        v->reqs.erase(it);
        return sfail(s, msg);
    }
    for (int k = 0; k < r->nbins; ++k) {
        if (ion_counts) ion_counts[k] = r->ion[static_cast<size_t>(k)];
        if (el_counts) el_counts[k] = r->el[static_cast<size_t>(k)];
    }
    if (energy)
        for (int k = 0; k < 6; ++k) energy[k] = r->energy[k];
    if (latency_s) *latency_s = r->latency;
    v->reqs.erase(it);
    return PIC_OK;
}

pic_status pic_server_set_policy(pic_server* v, int policy, int64_t max_resident_particles) {
    if (!v) return sfail(PIC_ERR_INVALID_ARG, "server is NULL");
    if (policy != PIC_SERVE_FIFO && policy != PIC_SERVE_SHORTEST_FIRST)
        return sfail(PIC_ERR_INVALID_ARG, "unknown policy");
    if (max_resident_particles < 0) return sfail(PIC_ERR_INVALID_ARG, "max_resident_particles must be >= 0");
    std::lock_guard<std::mutex> lk(v->m);
    v->policy = policy;
    v->max_resident = max_resident_particles;
    v->cv_work.notify_one();
    return PIC_OK;
}

pic_status pic_server_cancel(pic_server* v, int64_t ticket) {
    if (!v) return sfail(PIC_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(v->m);
    auto it = v->reqs.find(ticket);
    if (it == v->reqs.end()) return sfail(PIC_ERR_INVALID_ARG, "unknown ticket");
    Request* r = it->second.get();
    if (r->state == QUEUED) {
        for (auto q = v->queue.begin(); q != v->queue.end(); ++q)
            if (*q == ticket) {
                v->queue.erase(q);
                break;
            }
        v->st.queued = static_cast<int64_t>(v->queue.size());
        r->state = FAILED;
        r->status = PIC_ERR_STATE;
        r->err = "cancelled";
        v->st.failed++;
        v->cv_done.notify_all();
        return PIC_OK;
    }
    if (r->state == RUNNING) {
        r->cancel = true;
        return PIC_OK;
    }
    return sfail(PIC_ERR_STATE, "request already finished");
}

pic_status pic_server_stats(pic_server* v, pic_server_stats_t* out) {
    if (!v || !out) return sfail(PIC_ERR_INVALID_ARG, "server and out must not be NULL");
    std::lock_guard<std::mutex> lk(v->m);
    *out = v->st;
    return PIC_OK;
}

const char* pic_server_last_error(const pic_server*) { return t_err.c_str(); }

pic_status pic_server_destroy(pic_server* v) {
    if (!v) return PIC_OK;
    {
        std::lock_guard<std::mutex> lk(v->m);
        v->stop = true;
    }
    v->cv_work.notify_all();
    if (v->worker.joinable()) v->worker.join();
    pic_batch_destroy(v->batch);
    delete v;
    return PIC_OK;
}

}  // extern "C"
