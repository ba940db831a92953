// ecc_serve.cpp -- request loop with admission control and continuous batching.
//
// Jobs (mixed sizes, dtypes, gray ranges and complexes) are submitted from
// any thread.  A scheduler thread admits queued jobs in arrival order while
// their device bytes (input copy for host images, output and accumulator
// rows) fit the HBM budget, groups admitted jobs with the same
// (dtype, lo, hi, complex) key, and, whenever one of the n_streams slots is
// free, launches up to max_batch of them with one ecc_compute_batch call on
// that slot's stream.  Jobs that arrive while other batches run are admitted
// as budget frees up and join the next launch, so work from many requests
// overlaps on the device (continuous batching).  A completion thread waits
// for each slot's event, copies results out, releases budget, records
// latency (completion - submission) and runs callbacks.
//
// The paper has no serving layer; this composes the batched path
// (ecc_compute_batch) with the copy/compute overlap of Sec. 3.4.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "ecc.h"
#include "ecc_internal.h"
#include "ecc_plan.h"

namespace ecc {
namespace {

using Clock = std::chrono::steady_clock;

struct Key {
    int32_t dtype, lo, hi, mode;
    bool operator<(const Key &o) const
    {
        return std::tie(dtype, lo, hi, mode) < std::tie(o.dtype, o.lo, o.hi, o.mode);
    }
    bool operator==(const Key &o) const
    {
        return dtype == o.dtype && lo == o.lo && hi == o.hi && mode == o.mode;
    }
};

struct Job {
    uint64_t ticket = 0;
    ecc_image img{};
    Geom geom{};
    bool host_input = false;
    Key key{};
    int64_t voxels = 0;
    int64_t bytes = 0;           // budget charge
    int64_t *out = nullptr;      // host destination (may be null)
    ecc_done_fn done = nullptr;
    void *user = nullptr;
    Clock::time_point t_submit;
    unsigned char *d_input = nullptr;  // device copy of a host image
    int32_t nbins() const { return key.hi - key.lo + 1; }
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done_ev = nullptr;
    std::map<Key, ecc_plan_t> plans;
    std::vector<std::unique_ptr<Job>> jobs;  // jobs of the launch in flight
    long long *d_ecc = nullptr;              // [max_batch * 65536]
    long long *h_ecc = nullptr;              // pinned mirror
    ecc_plan_t plan_in_flight = nullptr;
    bool busy = false;
    Clock::time_point t_launch;
};

}  // namespace
}  // namespace ecc

struct ecc_server_s {
    ecc_server_desc d{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_sched;   // new work, free slot or shutdown
    std::condition_variable cv_done;    // a job finished
    std::deque<std::unique_ptr<ecc::Job>> pending;   // submitted, not admitted
    std::vector<std::unique_ptr<ecc::Job>> admitted; // admitted, not launched
    std::unordered_map<uint64_t, ecc_status> finished;  // ticket -> status (until waited)
    std::vector<ecc::Slot> slots;
    uint64_t next_ticket = 1;
    int64_t budget_used = 0, budget_peak = 0;
    bool stopping = false, cancel = false;
    std::thread sched, completer;
    // stats
    std::vector<double> latencies_us;
    double voxels_done = 0;
    int64_t jobs_done = 0, launches = 0;
    std::chrono::steady_clock::time_point t_first;
    bool have_first = false;
    std::chrono::steady_clock::time_point t_last;
};

namespace ecc {
namespace {

// Jobs worth a launch of their own: 3D volumes of at least 2^23 voxels
// whose rows the TMA-staged kernel can load (16-byte aligned base and pitches).
bool big_volume(const Job &j)
{
    const Geom &g = j.geom;
    if (j.host_input)  // copied densely into a fresh (256-byte aligned) buffer
        return g.ndim == 3 && j.voxels >= (int64_t(1) << 23) && (g.nx * g.esize) % 16 == 0;
    return g.ndim == 3 && j.voxels >= (int64_t(1) << 23) && reinterpret_cast<uintptr_t>(g.data) % 16 == 0 &&
           g.pitch_y % 16 == 0 && g.pitch_z % 16 == 0;
}

int64_t job_bytes(const Job &j)
{
    const int64_t io = j.host_input ? j.voxels * j.geom.esize : 0;
    return io + 2 * int64_t(j.nbins()) * 8;
}

void finish_job(ecc_server_s *s, std::unique_ptr<Job> j, ecc_status st, const long long *h_row)
{
    if (st == ECC_OK && j->out && h_row) std::memcpy(j->out, h_row, sizeof(int64_t) * j->nbins());
    const auto now = Clock::now();
    if (j->done) j->done(j->ticket, st, j->user);
    std::lock_guard<std::mutex> lk(s->mu);
    s->budget_used -= j->bytes;
    s->finished[j->ticket] = st;
    if (st == ECC_OK) {
        s->latencies_us.push_back(std::chrono::duration<double, std::micro>(now - j->t_submit).count());
        s->voxels_done += (double)j->voxels;
        ++s->jobs_done;
        s->t_last = now;
    }
    s->cv_done.notify_all();
    s->cv_sched.notify_all();
}

ecc_plan_t plan_for(Slot &slot, const Key &k, int32_t max_batch, uint32_t flags)
{
    auto it = slot.plans.find(k);
    if (it != slot.plans.end()) return it->second;
    ecc_plan_desc pd{};
    pd.dtype = k.dtype;
    pd.lo = k.lo;
    pd.hi = k.hi;
    pd.complex_mode = k.mode;
    pd.max_images = max_batch;
    pd.max_voxels = int64_t(1) << 40;
    pd.flags = flags & ECC_FLAG_NO_RANGE_CHECK;
    ecc_plan_t p = nullptr;
    if (ecc_plan(&p, &pd) != ECC_OK) return nullptr;
    slot.plans[k] = p;
    return p;
}

// Launch the admitted jobs with key k (at most max_batch) on a free slot.
// Called with s->mu held; releases it around CUDA calls.
void launch_batch(ecc_server_s *s, std::unique_lock<std::mutex> &lk, Slot &slot)
{
    const Key k = s->admitted.front()->key;
    std::vector<std::unique_ptr<Job>> batch;
    for (auto it = s->admitted.begin(); it != s->admitted.end() && (int)batch.size() < s->d.max_batch;) {
        if ((*it)->key == k) {
            batch.push_back(std::move(*it));
            it = s->admitted.erase(it);
        } else {
            ++it;
        }
    }
    // large 3D volumes whose rows the TMA kernel can stage go last and run
    // on the single-image kernel; everything else shares one batched launch
    std::stable_partition(batch.begin(), batch.end(), [](const std::unique_ptr<Job> &j) { return !big_volume(*j); });
    slot.busy = true;
    lk.unlock();

    cudaSetDevice(s->device);
    ecc_status st = ECC_OK;
    ecc_plan_t plan = plan_for(slot, k, s->d.max_batch, s->d.flags);
    if (!plan) st = ECC_E_NOMEM;
    std::vector<ecc_image> descs(batch.size());
    for (size_t i = 0; i < batch.size() && st == ECC_OK; ++i) {
        Job &j = *batch[i];
        descs[i] = j.img;
        if (j.host_input) {
            // dense device copy of the host image
            cudaError_t e = cudaMallocAsync((void **)&j.d_input, (size_t)(j.voxels * j.geom.esize), slot.stream);
            const Geom &g = j.geom;
            if (e == cudaSuccess) {
                if (g.ndim == 3) {
                    for (int64_t z = 0; z < g.nz && e == cudaSuccess; ++z)
                        e = cudaMemcpy2DAsync(j.d_input + z * g.ny * g.nx * g.esize, g.nx * g.esize,
                                              g.data + z * g.pitch_z, g.pitch_y, g.nx * g.esize, g.ny,
                                              cudaMemcpyHostToDevice, slot.stream);
                } else {
                    e = cudaMemcpy2DAsync(j.d_input, g.nx * g.esize, g.data, g.pitch_y, g.nx * g.esize, g.ny,
                                          cudaMemcpyHostToDevice, slot.stream);
                }
            }
            if (e != cudaSuccess) {
                st = cuda_fail(e, "server: input copy");
                break;
            }
            descs[i].data = j.d_input;
            descs[i].row_pitch = 0;
            descs[i].slice_pitch = 0;
        }
    }
    const int32_t nb = k.hi - k.lo + 1;
    size_t n_small = 0;
    while (n_small < batch.size() && !big_volume(*batch[n_small])) ++n_small;
    // a lone small job takes the plain path: one launch with the scan fused
    // into the stencil, against the batch graph's three (work list,
    // persistent kernel, segmented scan) -- at the nominal rate most
    // launches carry one job, so this is their latency
    if (n_small == 1) n_small = 0;
    if (st == ECC_OK && n_small > 0)
        st = ecc_compute_batch(plan, (int32_t)n_small, descs.data(), reinterpret_cast<int64_t *>(slot.d_ecc),
                               slot.stream);
    for (size_t i = n_small; i < batch.size() && st == ECC_OK; ++i)
        st = ecc_compute(plan, &descs[i], reinterpret_cast<int64_t *>(slot.d_ecc + i * nb), nullptr, slot.stream);
    if (st == ECC_OK) {
        cudaError_t e = cudaMemcpyAsync(slot.h_ecc, slot.d_ecc, sizeof(long long) * nb * batch.size(),
                                        cudaMemcpyDeviceToHost, slot.stream);
        for (auto &j : batch)
            if (j->d_input && e == cudaSuccess) e = cudaFreeAsync(j->d_input, slot.stream);
        if (e == cudaSuccess) e = cudaEventRecord(slot.done_ev, slot.stream);
        if (e != cudaSuccess) st = cuda_fail(e, "server: launch");
    }
    if (st != ECC_OK) {
        cudaStreamSynchronize(slot.stream);
        for (auto &j : batch) {
            if (j->d_input) cudaFree(j->d_input);
            j->d_input = nullptr;
            finish_job(s, std::move(j), st, nullptr);
        }
        lk.lock();
        slot.busy = false;
        return;
    }
    lk.lock();
    slot.jobs = std::move(batch);
    slot.plan_in_flight = plan;
    slot.t_launch = Clock::now();
    ++s->launches;
}

void scheduler_main(ecc_server_s *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // admission in arrival order against the budget
        while (!s->pending.empty()) {
            Job &j = *s->pending.front();
            if (s->cancel) {
                auto job = std::move(s->pending.front());
                s->pending.pop_front();
                s->finished[job->ticket] = ECC_E_CANCELLED;
                if (job->done) {
                    lk.unlock();
                    job->done(job->ticket, ECC_E_CANCELLED, job->user);
                    lk.lock();
                }
                s->cv_done.notify_all();
                continue;
            }
            if (s->budget_used + j.bytes > s->d.hbm_budget_bytes) break;
            s->budget_used += j.bytes;
            s->budget_peak = std::max(s->budget_peak, s->budget_used);
            s->admitted.push_back(std::move(s->pending.front()));
            s->pending.pop_front();
        }
        if (s->cancel) {
            for (auto &job : s->admitted) {
                s->budget_used -= job->bytes;
                s->finished[job->ticket] = ECC_E_CANCELLED;
                if (job->done) {
                    lk.unlock();
                    job->done(job->ticket, ECC_E_CANCELLED, job->user);
                    lk.lock();
                }
            }
            s->admitted.clear();
            s->cv_done.notify_all();
        }
        // dispatch onto free slots
        bool launched = false;
        for (auto &slot : s->slots) {
            if (s->admitted.empty()) break;
            if (slot.busy) continue;
            launch_batch(s, lk, slot);
            launched = true;
        }
        if (launched) {
            // the completion thread may be asleep with no slot busy: wake it
            // so the new launch's completion is seen when it happens, not at
            // the end of its idle wait
            s->cv_sched.notify_all();
            continue;
        }
        if (s->stopping && s->pending.empty() && s->admitted.empty()) {
            bool any_busy = false;
            for (auto &slot : s->slots) any_busy = any_busy || slot.busy;
            if (!any_busy) break;
        }
        s->cv_sched.wait_for(lk, std::chrono::milliseconds(2));
    }
}

void completer_main(ecc_server_s *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        bool idle = true;
        for (auto &slot : s->slots) {
            {
                std::lock_guard<std::mutex> g(s->mu);
                if (!slot.busy || slot.jobs.empty()) continue;
            }
            idle = false;
            if (cudaEventQuery(slot.done_ev) == cudaErrorNotReady) continue;
            ecc_status st = ecc_status_get(slot.plan_in_flight, slot.stream);
            std::vector<std::unique_ptr<Job>> jobs;
            {
                std::lock_guard<std::mutex> g(s->mu);
                jobs = std::move(slot.jobs);
                slot.jobs.clear();
            }
            for (size_t i = 0; i < jobs.size(); ++i) {
                const int32_t nb = jobs[i]->nbins();
                finish_job(s, std::move(jobs[i]), st, slot.h_ecc + i * nb);
            }
            std::lock_guard<std::mutex> g(s->mu);
            slot.busy = false;
            s->cv_sched.notify_all();
        }
        if (idle) {
            std::unique_lock<std::mutex> lk(s->mu);
            bool any_busy = false;
            for (auto &slot : s->slots) any_busy = any_busy || slot.busy;
            if (s->stopping && !any_busy && s->pending.empty() && s->admitted.empty()) break;
            s->cv_sched.wait_for(lk, std::chrono::microseconds(200));
        } else {
            std::this_thread::yield();
        }
    }
}

}  // namespace
}  // namespace ecc

using namespace ecc;

extern "C" {

ecc_status ecc_server_create(ecc_server_t *out, const ecc_server_desc *d)
{
    if (!out || !d) {
        set_error("ecc_server_create: NULL argument");
        return ECC_E_INVALID;
    }
    *out = nullptr;
    if (d->hbm_budget_bytes <= 0 || d->n_streams < 1 || d->n_streams > 64 || d->max_batch < 1 ||
        d->max_job_voxels < 1 || d->reserved) {
        set_error("ecc_server_create: invalid description");
        return ECC_E_INVALID;
    }
    auto *s = new ecc_server_s();
    s->d = *d;
    cudaGetDevice(&s->device);
    s->slots.resize(d->n_streams);
    for (auto &slot : s->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&slot.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&slot.done_ev, cudaEventDisableTiming);
        const size_t bytes = sizeof(long long) * (size_t)d->max_batch * 65536;
        if (e == cudaSuccess) e = cudaMalloc(&slot.d_ecc, bytes);
        if (e == cudaSuccess) e = cudaMallocHost(&slot.h_ecc, bytes);
        if (e != cudaSuccess) {
            ecc_status st = cuda_fail(e, "ecc_server_create");
            ecc_server_destroy(s, 1);
            return st;
        }
    }
    s->sched = std::thread(scheduler_main, s);
    s->completer = std::thread(completer_main, s);
    *out = s;
    return ECC_OK;
}

ecc_status ecc_server_prepare(ecc_server_t s, int32_t dtype, int32_t lo, int32_t hi, int32_t mode)
{
    if (!s) {
        set_error("ecc_server_prepare: NULL server");
        return ECC_E_INVALID;
    }
    const int32_t maxval = dtype == ECC_U8 ? 255 : 65535;
    if ((dtype != ECC_U8 && dtype != ECC_U16) || lo < 0 || hi < lo || hi > maxval ||
        (mode != ECC_VERTEX_MAX && mode != ECC_TOPCELL_MIN)) {
        set_error("ecc_server_prepare: invalid dtype, gray range or complex");
        return ECC_E_INVALID;
    }
    const Key k{dtype, lo, hi, mode};
    cudaSetDevice(s->device);
    for (auto &slot : s->slots) {
        {
            // hold the slot while its plan is made: the scheduler and the
            // completion thread skip a busy slot that has no jobs
            std::unique_lock<std::mutex> lk(s->mu);
            while (slot.busy) s->cv_sched.wait_for(lk, std::chrono::milliseconds(1));
            if (s->stopping) {
                set_error("ecc_server_prepare: the server is shutting down");
                return ECC_E_SHUTDOWN;
            }
            slot.busy = true;
        }
        ecc_plan_t plan = plan_for(slot, k, s->d.max_batch, s->d.flags);
        ecc_status st = plan ? prepare_batch(plan) : ECC_E_NOMEM;
        {
            std::lock_guard<std::mutex> g(s->mu);
            slot.busy = false;
            s->cv_sched.notify_all();
        }
        if (st != ECC_OK) return st;
    }
    return ECC_OK;
}

ecc_status ecc_submit(ecc_server_t s, const ecc_image *img, int32_t host_input, int32_t lo, int32_t hi,
                      int32_t mode, int64_t *out_ecc, ecc_done_fn done, void *user, uint64_t *ticket_out)
{
    if (!s || !img || !ticket_out) {
        set_error("ecc_submit: NULL argument");
        return ECC_E_INVALID;
    }
    auto j = std::make_unique<Job>();
    int64_t nv = 0;
    ecc_status st = image_geom(img, 0, s->d.max_job_voxels, &j->geom, &nv, false);
    if (st != ECC_OK) return st == ECC_E_BUSY ? ECC_E_INVALID : st;
    const int64_t maxval = img->dtype == ECC_U8 ? 255 : 65535;
    if (hi < lo || lo < 0 || hi > maxval || (mode != ECC_VERTEX_MAX && mode != ECC_TOPCELL_MIN)) {
        set_error("ecc_submit: invalid gray range or complex");
        return ECC_E_INVALID;
    }
    j->img = *img;
    j->host_input = host_input != 0;
    j->key = Key{img->dtype, lo, hi, mode};
    j->voxels = nv;
    j->bytes = job_bytes(*j);
    j->out = out_ecc;
    j->done = done;
    j->user = user;
    j->t_submit = Clock::now();
    if (j->bytes > s->d.hbm_budget_bytes) {
        set_error("ecc_submit: the job alone exceeds the HBM budget");
        return ECC_E_NOMEM;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) {
        set_error("ecc_submit: server is shutting down");
        return ECC_E_SHUTDOWN;
    }
    j->ticket = s->next_ticket++;
    *ticket_out = j->ticket;
    if (!s->have_first) {
        s->have_first = true;
        s->t_first = j->t_submit;
    }
    s->pending.push_back(std::move(j));
    s->cv_sched.notify_all();
    return ECC_OK;
}

ecc_status ecc_wait(ecc_server_t s, uint64_t ticket, int64_t timeout_us)
{
    if (!s) {
        set_error("ecc_wait: NULL server");
        return ECC_E_INVALID;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    if (ticket == 0 || ticket >= s->next_ticket) {
        set_error("ecc_wait: unknown ticket");
        return ECC_E_INVALID;
    }
    auto ready = [&] { return s->finished.count(ticket) != 0; };
    if (timeout_us < 0) {
        s->cv_done.wait(lk, ready);
    } else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
        set_error("ecc_wait: timed out");
        return ECC_E_TIMEOUT;
    }
    ecc_status st = s->finished[ticket];
    s->finished.erase(ticket);
    return st;
}

ecc_status ecc_server_stats(ecc_server_t s, double *out, int32_t n_out, int32_t reset)
{
    if (!s || !out || n_out < 0) {
        set_error("ecc_server_stats: invalid argument");
        return ECC_E_INVALID;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    std::vector<double> lat = s->latencies_us;
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double q) {
        if (lat.empty()) return 0.0;
        size_t i = (size_t)std::min<double>(lat.size() - 1, std::max(0.0, q * lat.size() - 1e-9));
        return lat[i];
    };
    const double busy =
        s->have_first ? std::chrono::duration<double, std::micro>(s->t_last - s->t_first).count() : 0.0;
    const double vals[8] = {(double)s->jobs_done, s->voxels_done, pct(0.50), pct(0.99),
                            lat.empty() ? 0.0 : lat.back(), (double)s->launches, busy, (double)s->budget_peak};
    for (int i = 0; i < n_out && i < 8; ++i) out[i] = vals[i];
    if (reset) {
        s->latencies_us.clear();
        s->voxels_done = 0;
        s->jobs_done = 0;
        s->launches = 0;
        s->have_first = false;
        s->budget_peak = s->budget_used;
    }
    return ECC_OK;
}

ecc_status ecc_server_destroy(ecc_server_t s, int32_t cancel)
{
    if (!s) {
        set_error("ecc_server_destroy: NULL server");
        return ECC_E_INVALID;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
        s->cancel = cancel != 0;
        s->cv_sched.notify_all();
    }
    if (s->sched.joinable()) s->sched.join();
    if (s->completer.joinable()) s->completer.join();
    cudaSetDevice(s->device);
    for (auto &slot : s->slots) {
        if (slot.stream) cudaStreamSynchronize(slot.stream);
        for (auto &kv : slot.plans) ecc_plan_destroy(kv.second);
        if (slot.d_ecc) cudaFree(slot.d_ecc);
        if (slot.h_ecc) cudaFreeHost(slot.h_ecc);
        if (slot.done_ev) cudaEventDestroy(slot.done_ev);
        if (slot.stream) cudaStreamDestroy(slot.stream);
    }
    delete s;
    return ECC_OK;
}

}  // extern "C"
