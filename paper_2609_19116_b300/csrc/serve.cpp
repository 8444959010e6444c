// Serving loop: sampling jobs for different circuits and noise rates arrive while others run.
//
// A job is pre-screened as a whole (Sec. 4.2), then its surviving shots are cut into chunks.
// Worker threads, one per CUDA stream, take the next chunk of the admitted job with the smallest
// aged remaining work (remaining work divided by 1 + age / 1 s, age counted from submission; a job
// older than 2 s goes before every younger one, oldest first), so small jobs do not queue behind
// large ones and no job waits unboundedly: under any load a job is at most 2 s from being served
// in submission order.  Chunks of different jobs run concurrently on the device, each as its
// own persistent engine launch on its worker's stream; inside a chunk the engine retires rejected
// shots early and back-fills their slots (Sec. 4.3).  A chunk is launched only when its in-flight
// footprint (slots x bytes of one slot of the capacity bucket the engine allocates) fits the HBM
// budget next to the chunks already running; finished chunks release their share.  Job buffers
// are stream-ordered (cudaMallocAsync / cudaFreeAsync), so no worker synchronises the device.
// Latency is measured from submission to the end of the job's last chunk.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <thread>

#include "qc_internal.h"

namespace qc {
namespace {

constexpr int WBINS = 16;
constexpr uint64_t CHUNK_SHOTS = 512;  // bounds how long a worker stays on one job
// A chunk holds at most this many shots per slot it is given: when the budget is nearly spent, a chunk
// shrinks with its slots instead of queueing hundreds of shots behind one or two of them (its latency
// stays about this many shot times, and the rest of the job waits for memory to free up).
constexpr uint64_t CHUNK_ROUNDS = 2;

struct Job {
    uint64_t id;
    CircuitImpl* circ;
    qc_noise noise;
    qc_mps_params prm;
    uint64_t shot0, nshots;
    int state = QC_PENDING;   // QC_PENDING, QC_OK, or an error
    bool prescreened = false, prescreening = false, cancelled = false;
    uint64_t survivors = 0;
    uint64_t* surv_dev = nullptr;
    uint64_t next = 0;         // next survivor index to hand out
    uint64_t done = 0;         // survivors finished
    int inflight = 0;          // chunks running
    int pending_error = QC_OK; // a failed chunk's status, reported once the job's other chunks end
    uint64_t footprint = 0;    // bytes per in-flight shot
    qc_counts counts[WBINS] = {};
    double submit_ms = 0, start_ms = -1, end_ms = -1;
    char error[sizeof(((qc_job_result*)nullptr)->error)] = {};
};

constexpr double AGE_MS = 1000.0;      // remaining work is divided by 1 + age / AGE_MS
constexpr double STARVE_MS = 2000.0;   // jobs older than this go first, oldest first

}  // namespace

struct Server {
    qc_serve_cfg cfg;
    int device = 0;
    int max_slots = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Job*> order;          // admission order
    std::map<uint64_t, Job*> jobs;
    uint64_t next_id = 1;
    uint64_t inflight_bytes = 0;
    bool stop = false;
    std::vector<std::thread> workers;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

    double now_ms() const {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }

    // Ends a job; its survivor buffer is released in stream order on `s` when a worker finishes it
    // (every chunk reading it has completed on its own stream by then), else synchronously.
    void finish(Job* j, int state, cudaStream_t s = nullptr, bool have_stream = false) {
        j->state = state;
        j->end_ms = now_ms();
        if (j->surv_dev) {
            if (have_stream) cudaFreeAsync(j->surv_dev, s);
            else cudaFree(j->surv_dev);
            j->surv_dev = nullptr;
        }
    }

    static void note_error(Job* j) {
        if (!j->error[0]) snprintf(j->error, sizeof j->error, "%s", qc_last_error());
    }

    // Pick work under the lock: a job to pre-screen (admission order; it is cheap and tells the
    // job's size), else a chunk of the admitted job with the least remaining work that fits the
    // budget (shortest remaining work first: small jobs do not wait behind large ones).  Remaining
    // work = survivors not yet handed out x the circuit's site operations per shot.
    bool pick(Job*& job, bool& pre, uint64_t& first, uint64_t& count, uint64_t& bytes) {
        const uint64_t free_b = cfg.hbm_budget_bytes > inflight_bytes ? cfg.hbm_budget_bytes - inflight_bytes : 0;
        const double now = now_ms();
        Job* best = nullptr;
        double best_score = 0;
        bool best_starved = false;
        uint64_t best_slots = 0, best_count = 0;
        for (Job* j : order) {
            if (j->state != QC_PENDING || j->cancelled) continue;
            if (!j->prescreened) {
                if (j->prescreening) continue;
                j->prescreening = true;
                job = j; pre = true;
                return true;
            }
            if (j->next >= j->survivors) continue;
            const uint64_t avail = j->survivors - j->next;
            const uint64_t n = std::min<uint64_t>(avail, CHUNK_SHOTS);
            uint64_t slots = std::min<uint64_t>(n, (uint64_t)max_slots);
            const uint64_t fit = j->footprint ? free_b / j->footprint : slots;
            if (fit == 0) continue;  // wait until memory frees up
            const double age = now - j->submit_ms;
            const bool starved = age > STARVE_MS;
            // aged shortest-remaining-work: small jobs first, but age shrinks a job's score, and a job
            // past the starvation bound goes before every job that is not (oldest first among those)
            const double work = (double)avail * (double)std::max<int64_t>(1, j->circ->n_updates);
            const double score = starved ? -age : work / (1.0 + age / AGE_MS);
            if (!best || (starved && !best_starved) || (starved == best_starved && score < best_score)) {
                best = j;
                best_score = score;
                best_starved = starved;
                best_slots = std::min(slots, fit);
                best_count = std::min<uint64_t>(n, CHUNK_ROUNDS * best_slots);
            }
        }
        if (!best) return false;
        Job* j = best;
        const uint64_t n = best_count;
        job = j; pre = false;
        first = j->next;
        count = n;
        bytes = best_slots * j->footprint;
        j->next += n;
        j->inflight += 1;
        inflight_bytes += bytes;
        if (j->start_ms < 0) j->start_ms = now;
        return true;
    }

    void worker() {
        cudaSetDevice(device);
        cudaStream_t s;
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        unsigned long long* counts = nullptr;
        cudaMalloc(&counts, 3 * WBINS * sizeof(unsigned long long));
        for (;;) {
            Job* j = nullptr;
            bool pre = false;
            uint64_t first = 0, count = 0, bytes = 0;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait(lk, [&] { return stop || pick(j, pre, first, count, bytes); });
                if (stop && !j) break;
            }
            if (pre) {
                // whole-job pre-screen; n_w counts every drawn shot (Eq. estimators)
                uint64_t nwords = (j->nshots + 63) / 64;
                uint64_t* mask = nullptr;
                uint64_t* surv = nullptr;
                qc_status st = QC_OK;
                if (cudaMallocAsync((void**)&mask, std::max<uint64_t>(nwords, 1) * 8, s) != cudaSuccess ||
                    cudaMallocAsync((void**)&surv, std::max<uint64_t>(j->nshots, 1) * 8, s) != cudaSuccess)
                    st = fail(QC_ENOMEM, "job buffers of %llu shots", (unsigned long long)j->nshots);
                qc_survivors sv{surv, j->nshots, 0};
                uint64_t hd[WBINS] = {}, hk[WBINS] = {};
                if (st == QC_OK)
                    st = prescreen_run(*j->circ, j->noise, j->shot0, j->nshots, mask, &sv, hd, hk, WBINS - 1, s);
                // admission charges one slot of the capacity bucket the engine will allocate
                uint64_t fp = 0;
                if (st == QC_OK) st = bucket_footprint(*j->circ, j->noise, j->prm, s, &fp);
                if (mask) cudaFreeAsync(mask, s);
                std::lock_guard<std::mutex> lk(mu);
                j->prescreening = false;
                if (st != QC_OK) {
                    note_error(j);
                    if (surv) cudaFreeAsync(surv, s);
                    finish(j, st, s, true);
                } else {
                    j->prescreened = true;
                    j->surv_dev = surv;
                    j->survivors = sv.count;
                    j->footprint = fp;
                    for (int w = 0; w < WBINS; ++w) j->counts[w].n = hd[w];
                    if (j->cancelled) finish(j, QC_ECANCELLED, s, true);
                    else if (sv.count == 0) { if (j->start_ms < 0) j->start_ms = now_ms(); finish(j, QC_OK, s, true); }
                }
                cv.notify_all();
                continue;
            }
            // a chunk of survivors
            qc_status st = QC_OK;
            unsigned long long h[3 * WBINS] = {};
            if (cudaMemsetAsync(counts, 0, sizeof h, s) != cudaSuccess) st = fail(QC_EDEVICE, "memset of the chunk counters");
            const int slots = (int)std::max<uint64_t>(1, bytes / std::max<uint64_t>(1, j->footprint));
            if (st == QC_OK)
                st = engine_launch(*j->circ, j->noise, j->surv_dev + first, count, j->prm, counts, WBINS - 1, nullptr, s,
                                   slots, true);
            if (st == QC_OK) {
                cudaError_t e = cudaMemcpyAsync(h, counts, sizeof h, cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) st = cuda_fail(e, "engine chunk");
            }
            std::lock_guard<std::mutex> lk(mu);
            if (st != QC_OK) note_error(j);
            inflight_bytes -= bytes;
            j->inflight -= 1;
            j->done += count;
            for (int w = 0; w < WBINS; ++w) {
                j->counts[w].n_acc += h[3 * w + 1];
                j->counts[w].n_err += h[3 * w + 2];
            }
            if (j->state == QC_PENDING) {
                // a failed chunk stops the job from handing out more chunks; the job ends with that
                // status once no chunk of it is in flight (they still read its survivor buffer)
                if (st != QC_OK && j->pending_error == QC_OK) j->pending_error = st;
                if (j->pending_error != QC_OK) j->cancelled = true;
                if (j->inflight == 0) {
                    if (j->pending_error != QC_OK) finish(j, j->pending_error, s, true);
                    else if (j->cancelled) finish(j, QC_ECANCELLED, s, true);
                    else if (j->done == j->survivors) finish(j, QC_OK, s, true);
                }
            }
            cv.notify_all();
        }
        cudaFree(counts);
        cudaStreamDestroy(s);
    }
};

}  // namespace qc

struct qc_server {
    qc::Server srv;
};

using namespace qc;

extern "C" qc_status mps_serve_create(const qc_serve_cfg* cfg, qc_server** out) {
    if (!cfg || !out) return fail(QC_EINVAL, "null argument");
    *out = nullptr;
    std::unique_ptr<qc_server> sp(new qc_server());
    Server& s = sp->srv;
    s.cfg = *cfg;
    QC_CUDA(cudaGetDevice(&s.device));
    int nsm = 0;
    QC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s.device));
    s.max_slots = cfg->max_slots > 0 ? cfg->max_slots : 16 * nsm;
    const int ns = cfg->n_streams > 0 ? cfg->n_streams : 64;
    for (int i = 0; i < ns; ++i) s.workers.emplace_back([&s] { s.worker(); });
    *out = sp.release();
    return QC_OK;
}

extern "C" qc_status mps_serve_submit(qc_server* server, const qc_circuit* circuit, qc_noise noise,
                                      qc_mps_params params, uint64_t shot0, uint64_t nshots, uint64_t* job_id) {
    if (!server || !circuit || !job_id) return fail(QC_EINVAL, "null argument");
    if (shot0 % 64) return fail(QC_EINVAL, "shot0 must be a multiple of 64");
    if (noise.fault_weight >= 0) return fail(QC_EINVAL, "the serving loop takes Bernoulli noise");
    if (params.chi_max < 1 || !(params.cutoff >= 0) || !(noise.p >= 0 && noise.p < 1))
        return fail(QC_EINVAL, "bad parameters");
    Server& s = server->srv;
    Job* j = new Job();
    j->circ = &const_cast<qc_circuit*>(circuit)->impl;
    j->noise = noise;
    j->prm = params;
    j->shot0 = shot0;
    j->nshots = nshots;
    {
        std::lock_guard<std::mutex> lk(s.mu);
        j->id = s.next_id++;
        j->submit_ms = s.now_ms();
        s.jobs[j->id] = j;
        s.order.push_back(j);
    }
    s.cv.notify_all();
    *job_id = j->id;
    return QC_OK;
}

extern "C" qc_status mps_serve_poll(qc_server* server, uint64_t job_id, qc_job_result* out) {
    if (!server || !out) return fail(QC_EINVAL, "null argument");
    Server& s = server->srv;
    std::lock_guard<std::mutex> lk(s.mu);
    auto it = s.jobs.find(job_id);
    if (it == s.jobs.end()) return fail(QC_EINVAL, "unknown job %llu", (unsigned long long)job_id);
    Job* j = it->second;
    if (j->state == QC_PENDING) return QC_PENDING;
    out->state = j->state;
    out->shots = j->nshots;
    out->survivors = j->survivors;
    for (int w = 0; w < WBINS; ++w) out->counts[w] = j->counts[w];
    out->submit_ms = j->submit_ms;
    out->start_ms = j->start_ms;
    out->end_ms = j->end_ms;
    memcpy(out->error, j->error, sizeof out->error);
    out->error[sizeof out->error - 1] = 0;
    return QC_OK;
}

extern "C" qc_status mps_serve_cancel(qc_server* server, uint64_t job_id) {
    if (!server) return fail(QC_EINVAL, "null argument");
    Server& s = server->srv;
    std::lock_guard<std::mutex> lk(s.mu);
    auto it = s.jobs.find(job_id);
    if (it == s.jobs.end()) return fail(QC_EINVAL, "unknown job");
    Job* j = it->second;
    if (j->state != QC_PENDING) return QC_OK;
    j->cancelled = true;
    if (j->inflight == 0 && !j->prescreening) s.finish(j, QC_ECANCELLED);
    s.cv.notify_all();
    return QC_OK;
}

extern "C" void mps_serve_destroy(qc_server* server) {
    if (!server) return;
    Server& s = server->srv;
    {
        std::lock_guard<std::mutex> lk(s.mu);
        s.stop = true;
        for (Job* j : s.order)
            if (j->state == QC_PENDING) j->cancelled = true;
    }
    s.cv.notify_all();
    for (auto& t : s.workers) t.join();
    for (auto& kv : s.jobs) {
        if (kv.second->surv_dev) cudaFree(kv.second->surv_dev);
        delete kv.second;
    }
    delete server;
}
