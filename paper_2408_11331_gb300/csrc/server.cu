// The served form: a request loop that keeps consensus jobs resident on the
// GPU and batches their sweeps (continuous batching).
//
// Submitted jobs wait in arrival order.  Each call of cc_server_progress
//   1. polls the contexts in flight; when a context's current graph launch has
//      ended, every job of it that has stopped is released at once (its
//      labels renumbered on the device and copied into the job's output
//      buffer, objective and sweep count recorded), without waiting for the
//      other jobs of its context; then the next launch is queued, or, once
//      all of its jobs have stopped, the context's memory goes back to the
//      server's pool;
//      Waiting jobs of the context's lane bin that fit the place of a
//      released job (no more vertices, CSR entries, partitions and label
//      rows) are loaded into it before the next launch, so they join the
//      running union between two graph launches (iteration-level batching);
//      a context whose jobs have all stopped is kept for such jobs too;
//   2. admits waiting jobs while a context slot is free and the device bytes
//      of the new context (computed exactly from the job sizes before
//      anything is allocated) fit in what the budget has left.  The oldest
//      waiting job opens the new context; later waiting jobs join it in
//      arrival order if they fall in the same lane bin (the number of lanes
//      that score one move, set by k), have a size within a factor 4 of the
//      first job's n (a context finishes with its slowest job, so a small job
//      does not wait for a large one) and still fit.  The jobs of a context
//      run as one disjoint union in the same kernel launches, on the
//      context's own stream, so contexts admitted while others run overlap
//      with them on the device.  Streams of smaller contexts get a higher
//      priority: when contexts share the GPU, the thread blocks of short jobs
//      are scheduled first, which keeps their latency close to running alone.
// Every job's results are those of running it alone (the sweep of a union is
// per-job exact), so results do not depend on the mix it was served in.
#include <algorithm>
#include <chrono>
#include <deque>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "context.cuh"

using namespace ccg;

namespace {

struct ServerJob {
    int64_t ticket;
    JobInput in;
    int32_t* out;  // caller's labels buffer (host, n entries)
    int bin;       // lane bin of k
};

struct Flight {
    cc_ctx* ctx = nullptr;
    std::vector<ServerJob> jobs;
    std::vector<char> released;  // per job: labels and record delivered
    int bin = 0;                 // lane bin of the context's jobs
    size_t bytes = 0;  // device bytes held by the context (persistent part of its plan)
    int slot = 0;      // pinned control-block slot
};

struct Record {
    int32_t done = 0;
    int32_t status = 0;
    int64_t F = 0;
    int32_t sweeps = 0;
};

thread_local std::string g_server_error;

}  // namespace

struct cc_server {
    cc_server_options sopt{};
    cc_options opt{};
    int device = 0;
    cudaMemPool_t pool = nullptr;
    DevState* pinned = nullptr;  // max_active control-block slots
    JobState* pinned_jobs = nullptr;  // max_active x max_batch_jobs job records
    std::vector<int> free_slots;
    std::deque<ServerJob> queue;
    std::vector<Flight> flights;
    std::unordered_map<int64_t, Record> records;
    std::deque<int64_t> finished;  // done, not yet reported by progress
    int64_t next_ticket = 0;
    size_t in_use = 0;
    int prio_least = 0, prio_greatest = 0;  // CUDA stream priority range (greatest is the lowest number)
    cc_server_info info{};
    std::string err;
};

namespace {

cc_status sfail(cc_server* s, cc_status code, const std::string& msg)
{
    if (s) s->err = msg;
    else g_server_error = msg;
    return code;
}

// Plan totals of one job (no checks beyond those of plan_jobs).
Plan job_totals(const JobInput& q)
{
    Plan p;
    p.jobs = 1;
    p.n = q.n;
    p.nnz = q.nnz;
    p.rows = (long long)q.n * ((q.k + 3) & ~3);
    p.keys = (long long)q.n * q.k;
    p.parts = q.k;
    p.kmax = q.k;
    return p;
}

void add_totals(Plan& a, const Plan& b)
{
    a.jobs += b.jobs;
    a.n += b.n;
    a.nnz += b.nnz;
    a.rows += b.rows;
    a.keys += b.keys;
    a.parts += b.parts;
    a.kmax = std::max(a.kmax, b.kmax);
}

size_t peak_bytes(Plan p, const cc_options& opt)
{
    finish_plan(p, opt);
    return p.persistent + p.temporary;
}

void finish_job(cc_server* s, const ServerJob& j, cc_status st, long long F, int sweeps)
{
    Record& r = s->records[j.ticket];
    r.done = 1;
    r.status = st;
    r.F = F;
    r.sweeps = sweeps;
    s->finished.push_back(j.ticket);
    s->info.completed += 1;
    if (st != CC_OK) s->info.failed += 1;
}

void release(cc_server* s, size_t idx)
{
    Flight& f = s->flights[idx];
    ctx_destroy(f.ctx);
    s->in_use -= f.bytes;
    s->free_slots.push_back(f.slot);
    s->flights.erase(s->flights.begin() + (long)idx);
}

JobState* flight_jobs(cc_server* s, const Flight& f)
{
    return s->pinned_jobs + (size_t)f.slot * (size_t)s->sopt.max_batch_jobs;
}

// Releases job j of a context whose run has stopped it: its labels alone
// (renumbered on the device, copied into its buffer), then its record.
// Returns 1 if a job was released.
int release_job(cc_server* s, Flight& f, size_t j)
{
    if (f.released[j]) return 0;
    const JobState& js = flight_jobs(s, f)[j];
    cc_status st = ctx_job_labels_now(f.ctx, (int)j, f.jobs[j].out);
    if (st != CC_OK) s->err = cc_last_error(f.ctx);
    finish_job(s, f.jobs[j], st, st == CC_OK ? js.F : 0, st == CC_OK ? js.sweeps : 0);
    f.released[j] = 1;
    return 1;
}

// Loads waiting jobs into the places of released jobs of flight f (in
// arrival order, first fit within a bounded look-ahead); returns how many.
int refill(cc_server* s, Flight& f)
{
    int loaded = 0;
    const int bin = f.jobs.empty() ? -1 : f.bin;
    for (size_t j = 0; j < f.jobs.size() && !s->queue.empty(); ++j) {
        if (!f.released[j]) continue;
        const size_t look = std::min(s->queue.size(), (size_t)64);
        for (size_t q = 0; q < look; ++q) {
            const ServerJob& w = s->queue[q];
            if (w.bin != bin || !ctx_slot_fits(f.ctx, (int)j, w.in)) continue;
            const ServerJob job = w;
            s->queue.erase(s->queue.begin() + (long)q);
            const cc_status st = ctx_load_job(f.ctx, (int)j, job.in);
            if (st != CC_OK) {
                s->err = cc_last_error(f.ctx);
                finish_job(s, job, st, 0, 0);
                if (st != CC_ERR_INVALID) return loaded;  // the context is no longer usable
                break;
            }
            f.jobs[j] = job;
            f.released[j] = 0;
            ++loaded;
            s->info.admitted += 1;
            s->info.admitted_running += 1;
            break;
        }
    }
    return loaded;
}

// Harvest of a finished context: every job not released yet, then the
// context's memory.
void harvest(cc_server* s, size_t idx)
{
    Flight& f = s->flights[idx];
    for (size_t j = 0; j < f.jobs.size(); ++j) release_job(s, f, j);
    release(s, idx);
}

// Polls every context in flight; returns how many jobs finished.
int poll_flights(cc_server* s)
{
    int finished = 0;
    for (size_t i = 0; i < s->flights.size();) {
        cc_status st = CC_OK;
        Flight& f = s->flights[i];
        const int r = ctx_async_poll_step(f.ctx, &st);
        if (r == 0) {
            ++i;
            continue;
        }
        if (r == 2) {
            // a launch ended and the run goes on: release the jobs that
            // stopped, then queue the next launch
            const JobState* js = flight_jobs(s, f);
            for (size_t j = 0; j < f.jobs.size(); ++j)
                if (js[j].stop) finished += release_job(s, f, j);
            refill(s, f);
            st = ctx_async_continue(f.ctx);
            if (st == CC_OK) {
                ++i;
                continue;
            }
            s->err = cc_last_error(f.ctx);
            for (size_t j = 0; j < f.jobs.size(); ++j)
                if (!f.released[j]) finish_job(s, f.jobs[j], st, 0, 0);
            release(s, i);
            continue;
        }
        if (r == 1) {
            // every job has stopped: release them; if waiting jobs fit their
            // places, the context goes on with those
            for (size_t j = 0; j < f.jobs.size(); ++j) finished += release_job(s, f, j);
            if (refill(s, f) > 0) {
                st = ctx_async_continue(f.ctx);
                if (st == CC_OK) {
                    ++i;
                    continue;
                }
                s->err = cc_last_error(f.ctx);
                for (size_t j = 0; j < f.jobs.size(); ++j)
                    if (!f.released[j]) finish_job(s, f.jobs[j], st, 0, 0);
            }
            release(s, i);
            continue;
        } else {
            s->err = cc_last_error(f.ctx);
            for (size_t j = 0; j < f.jobs.size(); ++j)
                if (!f.released[j]) {
                    finish_job(s, f.jobs[j], st, 0, 0);
                    ++finished;
                }
            release(s, i);
        }
    }
    return finished;
}

// Stream priority of a context with the given work size (label rows plus CSR
// entries): the device's greatest priority up to 2^16, then one step lower
// per factor 8, down to its least priority.
int priority_for(const cc_server* s, double work)
{
    int level = 0;
    for (double w = 65536.0; w < work; w *= 8.0) ++level;
    const int p = s->prio_greatest + level;
    return p > s->prio_least ? s->prio_least : p;
}

// Admits waiting jobs into new contexts; returns how many jobs were admitted.
int admit(cc_server* s)
{
    int admitted = 0;
    const size_t budget = (size_t)s->sopt.budget_bytes;
    while (!s->queue.empty() && !s->free_slots.empty() && (int)s->flights.size() < s->sopt.max_active) {
        const ServerJob first = s->queue.front();
        Plan acc = job_totals(first.in);
        const size_t alone = peak_bytes(acc, s->opt);
        if (alone > budget) {
            s->queue.pop_front();
            s->err = "job needs more device memory than the server's budget";
            finish_job(s, first, CC_ERR_OOM, 0, 0);
            continue;
        }
        if (s->in_use + alone > budget) break;  // wait for memory
        std::vector<size_t> take{0};
        const size_t look = std::min(s->queue.size(), (size_t)s->sopt.max_batch_jobs * 4);
        for (size_t q = 1; q < look && (int)take.size() < s->sopt.max_batch_jobs; ++q) {
            const ServerJob& j = s->queue[q];
            if (j.bin != first.bin) continue;
            if ((long long)j.in.n > 4LL * first.in.n || 4LL * j.in.n < (long long)first.in.n) continue;
            Plan t = acc;
            add_totals(t, job_totals(j.in));
            if (t.n >= (1LL << 31) || s->in_use + peak_bytes(t, s->opt) > budget) continue;
            acc = t;
            take.push_back(q);
        }
        Flight f;
        f.jobs.reserve(take.size());
        for (size_t q : take) f.jobs.push_back(s->queue[q]);
        f.released.assign(f.jobs.size(), 0);
        f.bin = first.bin;
        for (size_t r = take.size(); r-- > 0;) s->queue.erase(s->queue.begin() + (long)take[r]);
        std::vector<JobInput> in;
        in.reserve(f.jobs.size());
        for (const ServerJob& j : f.jobs) in.push_back(j.in);
        Plan p = acc;
        finish_plan(p, s->opt);
        f.bytes = p.persistent;
        f.slot = s->free_slots.back();
        cc_status st = ctx_create((int)in.size(), in.data(), false, &s->opt, nullptr, s->pool, &f.ctx,
                                  priority_for(s, (double)acc.keys + (double)acc.nnz));
        if (st == CC_OK)
            st = ctx_async_start(f.ctx, s->opt.max_sweeps, s->pinned + f.slot,
                                 s->pinned_jobs + (size_t)f.slot * (size_t)s->sopt.max_batch_jobs);
        if (st != CC_OK) {
            s->err = f.ctx ? cc_last_error(f.ctx) : cc_last_error(nullptr);
            if (f.ctx) ctx_destroy(f.ctx);
            for (const ServerJob& j : f.jobs) finish_job(s, j, st, 0, 0);
            continue;
        }
        s->free_slots.pop_back();
        s->in_use += f.bytes;
        admitted += (int)f.jobs.size();
        s->info.batches += 1;
        s->info.admitted += (int64_t)f.jobs.size();
        s->flights.push_back(std::move(f));
        s->info.max_in_flight = std::max<int64_t>(s->info.max_in_flight, (int64_t)s->flights.size());
        s->info.peak_bytes = std::max<int64_t>(s->info.peak_bytes, (int64_t)s->in_use);
    }
    return admitted;
}

}  // namespace

extern "C" {

cc_status cc_plan_batches(int32_t jobs, const cc_job_desc* descs, const cc_options* opt, int64_t budget_bytes,
                          int32_t max_jobs, int32_t* batch_of, int32_t* batches)
{
    if (jobs < 1 || !descs || !batch_of || budget_bytes <= 0)
        return sfail(nullptr, CC_ERR_INVALID, "cc_plan_batches needs jobs >= 1, descriptors, output and a budget");
    const cc_options o = resolve_options(opt);
    std::string msg;
    cc_status r = check_options(o, &msg);
    if (r != CC_OK) return sfail(nullptr, r, msg);
    std::vector<JobInput> in(jobs);
    for (int j = 0; j < jobs; ++j) {
        in[j] = JobInput{descs[j].n, descs[j].nnz, descs[j].row_off, descs[j].col, descs[j].k, descs[j].labels};
        Plan p;
        r = plan_jobs(1, &in[j], o, &p, &msg);
        if (r != CC_OK) return sfail(nullptr, r, "job " + std::to_string(j) + ": " + msg);
    }
    // lane bins in increasing order, jobs in index order within a bin
    std::vector<int> order(jobs);
    for (int j = 0; j < jobs; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return lanes_for_k(in[x].k) < lanes_for_k(in[y].k); });
    const size_t budget = (size_t)budget_bytes;
    int nb = 0, open_bin = -1, count = 0;
    Plan acc;
    for (int j : order) {
        const Plan one = job_totals(in[j]);
        if (peak_bytes(one, o) > budget) {
            batch_of[j] = -1;
            continue;
        }
        const int bin = lanes_for_k(in[j].k);
        Plan t = acc;
        add_totals(t, one);
        const bool fits = open_bin == bin && (max_jobs <= 0 || count < max_jobs) && t.n < (1LL << 31) &&
                          peak_bytes(t, o) <= budget;
        if (!fits) {
            ++nb;
            open_bin = bin;
            count = 0;
            acc = one;
        } else {
            acc = t;
        }
        batch_of[j] = nb - 1;
        ++count;
    }
    if (batches) *batches = nb;
    return CC_OK;
}

void cc_server_default_options(cc_server_options* o)
{
    if (!o) return;
    *o = cc_server_options{};
    o->max_active = 8;
    o->max_batch_jobs = 256;
}

cc_status cc_server_create(const cc_server_options* sopt, const cc_options* opt, cc_server** out)
{
    if (!out) return sfail(nullptr, CC_ERR_INVALID, "out is NULL");
    *out = nullptr;
    cc_server_options so;
    cc_server_default_options(&so);
    if (sopt) so = *sopt;
    for (int r : so.reserved)
        if (r != 0) return sfail(nullptr, CC_ERR_INVALID, "reserved server option fields must be zero");
    if (so.budget_bytes < 0 || so.max_active < 0 || so.max_batch_jobs < 0)
        return sfail(nullptr, CC_ERR_INVALID, "server options must not be negative");
    if (so.max_active == 0) so.max_active = 8;
    if (so.max_active > 64) return sfail(nullptr, CC_ERR_INVALID, "max_active must be <= 64");
    if (so.max_batch_jobs == 0) so.max_batch_jobs = 256;
    const cc_options o = resolve_options(opt);
    std::string msg;
    cc_status r = check_options(o, &msg);
    if (r != CC_OK) return sfail(nullptr, r, msg);
    cc_server* s = new cc_server();
    s->opt = o;
    auto bail = [&](cudaError_t e, const char* what) {
        g_server_error = std::string(what) + ": " + cudaGetErrorString(e);
        if (s->pinned) cudaFreeHost(s->pinned);
        if (s->pinned_jobs) cudaFreeHost(s->pinned_jobs);
        if (s->pool) cudaMemPoolDestroy(s->pool);
        delete s;
        return e == cudaErrorMemoryAllocation ? CC_ERR_OOM : CC_ERR_CUDA;
    };
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) return bail(e, "cudaGetDevice");
    e = cudaDeviceGetStreamPriorityRange(&s->prio_least, &s->prio_greatest);
    if (e != cudaSuccess) return bail(e, "cudaDeviceGetStreamPriorityRange");
    if (so.budget_bytes == 0) {
        size_t free_b = 0, total_b = 0;
        e = cudaMemGetInfo(&free_b, &total_b);
        if (e != cudaSuccess) return bail(e, "cudaMemGetInfo");
        so.budget_bytes = (int64_t)(free_b / 10 * 8);
    }
    s->sopt = so;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->device;
    e = cudaMemPoolCreate(&s->pool, &props);
    if (e != cudaSuccess) return bail(e, "cudaMemPoolCreate");
    // keep up to the budget reserved between contexts instead of returning it
    // to the driver at every synchronisation
    uint64_t keep = (uint64_t)so.budget_bytes;
    e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) return bail(e, "cudaMemPoolSetAttribute");
    e = cudaHostAlloc(reinterpret_cast<void**>(&s->pinned), sizeof(DevState) * (size_t)so.max_active,
                      cudaHostAllocDefault);
    if (e != cudaSuccess) return bail(e, "cudaHostAlloc");
    e = cudaHostAlloc(reinterpret_cast<void**>(&s->pinned_jobs),
                      sizeof(JobState) * (size_t)so.max_active * (size_t)so.max_batch_jobs, cudaHostAllocDefault);
    if (e != cudaSuccess) return bail(e, "cudaHostAlloc");
    for (int i = so.max_active - 1; i >= 0; --i) s->free_slots.push_back(i);
    s->info.budget_bytes = so.budget_bytes;
    *out = s;
    return CC_OK;
}

cc_status cc_server_submit(cc_server* s, const cc_job_desc* job, int32_t* labels_out, int64_t* ticket)
{
    if (!s || !job || !labels_out) return sfail(s, CC_ERR_INVALID, "null argument");
    const JobInput in{job->n, job->nnz, job->row_off, job->col, job->k, job->labels};
    if (!in.row_off || !in.labels || (in.nnz > 0 && !in.col)) return sfail(s, CC_ERR_INVALID, "null input pointer");
    Plan p;
    std::string msg;
    cc_status r = plan_jobs(1, &in, s->opt, &p, &msg);
    if (r != CC_OK) return sfail(s, r, msg);
    ServerJob j{s->next_ticket++, in, labels_out, lanes_for_k(in.k)};
    s->records[j.ticket] = Record{};
    s->queue.push_back(j);
    s->info.submitted += 1;
    if (ticket) *ticket = j.ticket;
    return CC_OK;
}

cc_status cc_server_progress(cc_server* s, int32_t wait, int64_t* done, int32_t max_done, int32_t* n_done,
                             int64_t* pending)
{
    if (!s) return sfail(nullptr, CC_ERR_INVALID, "server is NULL");
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const int fin = poll_flights(s);
        const int adm = admit(s);
        if (!wait || fin > 0 || adm > 0 || !s->finished.empty() || s->flights.empty()) break;
        // a waiting call gives up after a second, so that a caller can always
        // submit new arrivals
        if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(1)) break;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    int32_t nd = 0;
    while (!s->finished.empty() && nd < max_done && done) {
        done[nd++] = s->finished.front();
        s->finished.pop_front();
    }
    if (n_done) *n_done = nd;
    if (pending) *pending = s->info.submitted - s->info.completed;
    return CC_OK;
}

cc_status cc_server_job(cc_server* s, int64_t ticket, int32_t* done, int64_t* F, int32_t* sweeps, int32_t* status)
{
    if (!s) return sfail(nullptr, CC_ERR_INVALID, "server is NULL");
    auto it = s->records.find(ticket);
    if (it == s->records.end()) return sfail(s, CC_ERR_INVALID, "unknown ticket");
    const Record& r = it->second;
    if (done) *done = r.done;
    if (F) *F = r.F;
    if (sweeps) *sweeps = r.sweeps;
    if (status) *status = r.status;
    return CC_OK;
}

cc_status cc_server_stats(const cc_server* s, cc_server_info* out)
{
    if (!s || !out) return sfail(nullptr, CC_ERR_INVALID, "null argument");
    *out = s->info;
    out->in_flight = (int64_t)s->flights.size();
    out->queued = (int64_t)s->queue.size();
    out->bytes_in_use = (int64_t)s->in_use;
    return CC_OK;
}

const char* cc_server_last_error(const cc_server* s)
{
    return s ? s->err.c_str() : g_server_error.c_str();
}

void cc_server_destroy(cc_server* s)
{
    if (!s) return;
    for (Flight& f : s->flights) {
        if (f.ctx && f.ctx->stream) cudaStreamSynchronize(f.ctx->stream);
        ctx_destroy(f.ctx);
    }
    s->flights.clear();
    cudaDeviceSynchronize();
    if (s->pinned) cudaFreeHost(s->pinned);
    if (s->pinned_jobs) cudaFreeHost(s->pinned_jobs);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
}

}  // extern "C"
