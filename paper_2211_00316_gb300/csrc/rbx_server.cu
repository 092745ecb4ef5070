// Served form: continuous batching of reconstruction requests on one GPU.
//
// Requests (geometry, initial model, frequency sweep, measured data, all host buffers)
// arrive at any time. A worker thread admits them in arrival order while their estimated
// device bytes fit the HBM budget and fewer than max_inflight run; each admitted request
// becomes a job with its own stream, its data and model resident on the device for its whole
// sweep, and its sweep queued at once. Jobs on different streams overlap on the device.
// Completed jobs are found by event query, their model and last-update scalars copied out,
// their memory released (stream-ordered, no device-wide synchronisation), which admits the
// next waiting requests. Latency is measured on the host from the moment rbx_server_submit is
// entered to completion. The server's mutex guards only the queues and the published state
// of each request: the worker takes a request off the queue under it, does the CUDA work
// (job creation, uploads, completion, release) without it, and publishes the outcome under
// it again, so a client's submit never waits behind device work.
#include "rbx_internal.cuh"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

using namespace rbx;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    long long id = 0;
    rbx_geometry g{};
    std::vector<float> c0;
    std::vector<double> freqs;
    std::vector<unsigned char> data;   // nf x N x N complex64
    // published state: read by clients, written under the server's mutex
    int state = RBX_REQ_QUEUED;
    rbx_status status = RBX_OK;
    std::string err;
    Clock::time_point t_submit, t_start, t_done;
    bool started = false;
    size_t bytes = 0;
    std::vector<float> c_out;
    rbx_stats last{};
    // the worker's own while the request runs (never touched by clients)
    rbx_status w_status = RBX_OK;
    std::string w_err;
    std::vector<float> w_c_out;
    rbx_stats w_last{};
    Clock::time_point w_done;
    rbx_job *job = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    void *d_data = nullptr, *d_c = nullptr;
};

}  // namespace

struct rbx_server {
    size_t budget = 0, used = 0;
    int max_inflight = 1;
    Clock::time_point t0 = Clock::now();
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    long long next_id = 1;
    std::map<long long, std::shared_ptr<Request>> reqs;
    std::deque<long long> pending;
    std::vector<long long> inflight;
};

static void release(Request &r)
{
    if (r.job) rbx_destroy(r.job);   // waits for the job's stream, frees its pool memory
    if (r.d_data) cudaFreeAsync(r.d_data, r.stream);
    if (r.d_c) cudaFreeAsync(r.d_c, r.stream);
    if (r.stream) cudaStreamSynchronize(r.stream);
    if (r.done) cudaEventDestroy(r.done);
    if (r.stream) cudaStreamDestroy(r.stream);
    r.job = nullptr;
    r.d_data = r.d_c = nullptr;
    r.done = nullptr;
    r.stream = nullptr;
    std::vector<unsigned char>().swap(r.data);
}

// Records a failure in the worker's private copy of the outcome (published by publish_end()).
static void fail_req(Request &r, rbx_status st, const std::string &msg)
{
    r.w_status = st;
    r.w_err = msg;
    r.w_done = Clock::now();
}

// Copies the worker's outcome of an ended request into its published state. Called with
// the server's mutex held.
static void publish_end(Request &r)
{
    r.status = r.w_status;
    r.err = r.w_err;
    r.t_done = r.w_done;
    r.last = r.w_last;
    r.c_out.swap(r.w_c_out);
    r.state = r.w_status == RBX_OK ? RBX_REQ_DONE : RBX_REQ_FAILED;
}

// Create the job, upload model and data, queue the sweep and its completion event. Runs
// without the server's mutex; the request is already off the queue (state RUNNING).
static bool start(Request &r)
{
    auto cuda_fail = [&](const char *what, cudaError_t e) {
        fail_req(r, RBX_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
        cudaGetLastError();
        return false;
    };
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&r.stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail("stream", e);
    if ((e = cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail("event", e);
    rbx_status st = rbx_create(&r.job, r.stream);
    if (st == RBX_OK) st = rbx_set_geometry(r.job, &r.g, nullptr);
    if (st != RBX_OK) {
        fail_req(r, st, r.job ? rbx_last_error(r.job) : "job creation failed");
        return false;
    }
    const size_t nxy = (size_t)r.g.nx * r.g.ny;
    if ((e = cudaMallocAsync(&r.d_c, nxy * sizeof(float), r.stream)) != cudaSuccess) return cuda_fail("model", e);
    if ((e = cudaMallocAsync(&r.d_data, r.data.size(), r.stream)) != cudaSuccess) return cuda_fail("data", e);
    if ((e = cudaMemcpyAsync(r.d_c, r.c0.data(), nxy * sizeof(float), cudaMemcpyHostToDevice, r.stream)) != cudaSuccess)
        return cuda_fail("model upload", e);
    if ((e = cudaMemcpyAsync(r.d_data, r.data.data(), r.data.size(), cudaMemcpyHostToDevice, r.stream)) != cudaSuccess)
        return cuda_fail("data upload", e);
    if ((st = rbx_set_model(r.job, static_cast<const float *>(r.d_c))) != RBX_OK) {
        fail_req(r, st, rbx_last_error(r.job));
        return false;
    }
    if ((st = job_enqueue_sweep(r.job, r.freqs.data(), (int)r.freqs.size(), r.d_data)) != RBX_OK) {
        fail_req(r, st, rbx_last_error(r.job));
        return false;
    }
    if ((e = cudaEventRecord(r.done, r.stream)) != cudaSuccess) return cuda_fail("completion event", e);
    return true;
}

// Read the finished sweep's scalars and model (no mutex held).
static void finish(Request &r)
{
    rbx_stats st{};
    rbx_status s = job_read_sweep(r.job, (int)r.freqs.size(), &st);
    const size_t nxy = (size_t)r.g.nx * r.g.ny;
    r.w_c_out.resize(nxy);
    cudaError_t e = cudaMemcpyAsync(r.w_c_out.data(), job_model(r.job), nxy * sizeof(float), cudaMemcpyDeviceToHost,
                                    r.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r.stream);
    r.w_done = Clock::now();
    r.w_last = st;
    if (s != RBX_OK) {
        fail_req(r, s, rbx_last_error(r.job));
    } else if (e != cudaSuccess) {
        fail_req(r, RBX_ECUDA, std::string("model download: ") + cudaGetErrorString(e));
    } else {
        r.w_status = RBX_OK;
    }
}

static void worker_loop(rbx_server *s)
{
    cudaSetDevice(s->device);
    // requests this worker runs; only the worker touches this list
    std::vector<std::shared_ptr<Request>> running;
    while (true) {
        bool progressed = false;
        // retire completed jobs: CUDA work unlocked, the outcome published under the mutex
        for (size_t k = 0; k < running.size();) {
            Request &r = *running[k];
            cudaError_t q = cudaEventQuery(r.done);
            if (q == cudaErrorNotReady) { ++k; continue; }
            if (q == cudaSuccess) finish(r);
            else fail_req(r, RBX_ECUDA, std::string("job failed: ") + cudaGetErrorString(q));
            release(r);
            {
                std::lock_guard<std::mutex> lk(s->mu);
                publish_end(r);
                s->used -= r.bytes;
                s->inflight.erase(std::find(s->inflight.begin(), s->inflight.end(), r.id));
            }
            running.erase(running.begin() + k);
            progressed = true;
        }
        // admit waiting requests in arrival order while they fit: take one off the queue
        // under the mutex, start it without the mutex
        while (true) {
            std::shared_ptr<Request> rp;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                if (s->stop || s->pending.empty() || (int)s->inflight.size() >= s->max_inflight) break;
                Request &r = *s->reqs[s->pending.front()];
                if (r.bytes > s->budget) {
                    r.w_status = RBX_ENOMEM;
                    r.w_err = "request needs more device memory than the server's budget";
                    r.w_done = Clock::now();
                    publish_end(r);
                    s->pending.pop_front();
                    progressed = true;
                    s->cv.notify_all();
                    continue;
                }
                if (s->used + r.bytes > s->budget) break;
                s->pending.pop_front();
                s->used += r.bytes;
                s->inflight.push_back(r.id);
                r.state = RBX_REQ_RUNNING;   // no longer cancellable; the worker owns its buffers
                r.started = true;
                r.t_start = Clock::now();
                rp = s->reqs[r.id];
            }
            progressed = true;
            if (start(*rp)) {
                running.push_back(rp);
            } else {
                release(*rp);
                std::lock_guard<std::mutex> lk(s->mu);
                publish_end(*rp);
                s->used -= rp->bytes;
                s->inflight.erase(std::find(s->inflight.begin(), s->inflight.end(), rp->id));
            }
        }
        std::unique_lock<std::mutex> lk(s->mu);
        if (progressed) s->cv.notify_all();
        if (s->stop && running.empty()) break;
        s->cv.wait_for(lk, std::chrono::microseconds(progressed ? 0 : 200));
    }
    std::lock_guard<std::mutex> lk(s->mu);
    for (long long id : s->pending) {
        Request &r = *s->reqs[id];
        r.state = RBX_REQ_CANCELLED;
        r.status = RBX_ESTATE;
        r.err = "server stopped before the request ran";
    }
    s->pending.clear();
    s->cv.notify_all();
}

extern "C" {

size_t rbx_estimate_bytes(const rbx_geometry *geom, int nf)
{
    if (!geom || nf < 1) return 0;
    return job_bytes_estimate(*geom, nf);
}

rbx_status rbx_server_create(rbx_server **out, size_t hbm_budget_bytes, int max_inflight)
{
    if (!out || hbm_budget_bytes == 0 || max_inflight < 1) return RBX_EINVAL;
    *out = nullptr;
    rbx_server *s = new (std::nothrow) rbx_server();
    if (!s) return RBX_ENOMEM;
    s->budget = hbm_budget_bytes;
    s->max_inflight = max_inflight;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return RBX_ECUDA;
    }
    try {
        s->worker = std::thread(worker_loop, s);
    } catch (...) {
        delete s;
        return RBX_ENOMEM;
    }
    *out = s;
    return RBX_OK;
}

rbx_status rbx_server_submit(rbx_server *s, const rbx_geometry *g, const float *c_init_host, const double *freqs_host,
                             int nf, const void *data_host, long long *ticket)
{
    // latency counts from here: the copies of the inputs below are part of it
    const Clock::time_point t_call = Clock::now();
    if (!s || !g || !c_init_host || !freqs_host || !data_host || !ticket || nf < 1) return RBX_EINVAL;
    if (g->nx < 1 || g->ny < 1 || g->n_xducers < 1 || nf > kHistSlots) return RBX_EINVAL;
    auto r = std::make_shared<Request>();
    r->t_submit = t_call;
    r->g = *g;
    const size_t nxy = (size_t)g->nx * g->ny, nn = (size_t)g->n_xducers * g->n_xducers;
    try {
        r->c0.assign(c_init_host, c_init_host + nxy);
        r->freqs.assign(freqs_host, freqs_host + nf);
        const unsigned char *d = static_cast<const unsigned char *>(data_host);
        r->data.assign(d, d + (size_t)nf * nn * 8);
    } catch (...) {
        return RBX_ENOMEM;
    }
    r->bytes = job_bytes_estimate(*g, nf);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return RBX_ESTATE;
    r->id = s->next_id++;
    s->reqs[r->id] = r;
    s->pending.push_back(r->id);
    *ticket = r->id;
    s->cv.notify_all();
    return RBX_OK;
}

rbx_status rbx_server_poll(rbx_server *s, long long ticket, int *state, double *latency_s, float *c_out_host,
                           rbx_stats *last)
{
    if (!s) return RBX_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return RBX_EINVAL;
    Request &r = *it->second;
    if (state) *state = r.state;
    bool ended = r.state == RBX_REQ_DONE || r.state == RBX_REQ_FAILED || r.state == RBX_REQ_CANCELLED;
    if (ended && latency_s) *latency_s = std::chrono::duration<double>(r.t_done - r.t_submit).count();
    if (r.state == RBX_REQ_DONE) {
        if (c_out_host) std::memcpy(c_out_host, r.c_out.data(), r.c_out.size() * sizeof(float));
        if (last) *last = r.last;
    }
    return ended ? r.status : RBX_OK;
}

rbx_status rbx_server_wait(rbx_server *s, long long ticket, double timeout_s)
{
    if (!s) return RBX_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return RBX_EINVAL;
    std::shared_ptr<Request> r = it->second;
    auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    bool ok = s->cv.wait_until(lk, until, [&] {
        return r->state == RBX_REQ_DONE || r->state == RBX_REQ_FAILED || r->state == RBX_REQ_CANCELLED;
    });
    return ok ? r->status : RBX_ETIMEOUT;
}

rbx_status rbx_server_cancel(rbx_server *s, long long ticket)
{
    if (!s) return RBX_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return RBX_EINVAL;
    Request &r = *it->second;
    if (r.state != RBX_REQ_QUEUED) return RBX_ESTATE;
    for (auto p = s->pending.begin(); p != s->pending.end(); ++p)
        if (*p == ticket) {
            s->pending.erase(p);
            break;
        }
    r.state = RBX_REQ_CANCELLED;
    r.status = RBX_OK;
    r.t_done = Clock::now();
    std::vector<unsigned char>().swap(r.data);
    s->cv.notify_all();
    return RBX_OK;
}

rbx_status rbx_server_times(rbx_server *s, long long ticket, double *t_submit, double *t_start, double *t_end)
{
    if (!s) return RBX_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return RBX_EINVAL;
    const Request &r = *it->second;
    auto sec = [&](Clock::time_point t) { return std::chrono::duration<double>(t - s->t0).count(); };
    bool ended = r.state == RBX_REQ_DONE || r.state == RBX_REQ_FAILED || r.state == RBX_REQ_CANCELLED;
    if (t_submit) *t_submit = sec(r.t_submit);
    if (t_start) *t_start = r.started ? sec(r.t_start) : -1.0;
    if (t_end) *t_end = ended ? sec(r.t_done) : -1.0;
    return RBX_OK;
}

rbx_status rbx_server_info(rbx_server *s, int *queued, int *running, size_t *bytes_in_use)
{
    if (!s) return RBX_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (queued) *queued = (int)s->pending.size();
    if (running) *running = (int)s->inflight.size();
    if (bytes_in_use) *bytes_in_use = s->used;
    return RBX_OK;
}

const char *rbx_server_error(rbx_server *s, long long ticket)
{
    if (!s) return "null server";
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    return it == s->reqs.end() ? "unknown ticket" : it->second->err.c_str();
}

rbx_status rbx_server_destroy(rbx_server *s)
{
    if (!s) return RBX_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    delete s;
    return RBX_OK;
}

}  // extern "C"
