// The C ABI declared in include/cc.h: context lifetime (one job, or a batch of
// jobs held as one disjoint union), the sweep loop as captured CUDA graphs,
// and the output calls.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "context.cuh"

using namespace ccg;

namespace {

thread_local std::string g_create_error;

cc_status fail(cc_ctx* c, cc_status code, const std::string& msg)
{
    if (c) c->err = msg;
    else g_create_error = msg;
    return code;
}

cc_status cuda_fail(cc_ctx* c, cudaError_t e, const char* what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(c, CC_ERR_OOM, m);
    return fail(c, CC_ERR_CUDA, m);
}

#define CC_CUDA(c, expr)                                   \
    do {                                                   \
        cudaError_t e_ = (expr);                           \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #expr); \
    } while (0)

template <typename T>
cudaError_t dalloc(cc_ctx* c, T** p, size_t count)
{
    void* q = nullptr;
    const size_t bytes = count * sizeof(T) > 0 ? count * sizeof(T) : 16;
    cudaError_t e = c->pool ? cudaMallocFromPoolAsync(&q, bytes, c->pool, c->own_stream) : cudaMalloc(&q, bytes);
    if (e != cudaSuccess) return e;
    c->allocs.push_back(q);
    c->bytes += bytes;
    *p = static_cast<T*>(q);
    return cudaSuccess;
}

void destroy_graph(RunGraph& g)
{
    if (g.exec) cudaGraphExecDestroy(g.exec);
    for (cudaEvent_t e : g.bound) cudaEventDestroy(e);
    for (cudaEvent_t e : g.prop) cudaEventDestroy(e);
    g = RunGraph();
}

void free_all(cc_ctx* c)
{
    for (auto& kv : c->graphs) destroy_graph(kv.second);
    c->graphs.clear();
    if (c->pool) {
        // stream-ordered: the memory returns to the pool once the context's
        // queued work has finished, without waiting here
        if (c->stream != c->own_stream) {
            cudaEvent_t ev = nullptr;
            if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
                cudaEventRecord(ev, c->stream);
                cudaStreamWaitEvent(c->own_stream, ev, 0);
                cudaEventDestroy(ev);
            }
        }
        for (void* p : c->allocs) cudaFreeAsync(p, c->own_stream);
    } else {
        for (void* p : c->allocs) cudaFree(p);
    }
    c->allocs.clear();
    c->bytes = 0;
    if (c->chunk_done) cudaEventDestroy(c->chunk_done);
    c->chunk_done = nullptr;
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    c->own_stream = nullptr;
    if (c->body_stream) cudaStreamDestroy(c->body_stream);
    c->body_stream = nullptr;
    if (c->loop_stream) cudaStreamDestroy(c->loop_stream);
    c->loop_stream = nullptr;
}

unsigned long long next_pow2(unsigned long long x)
{
    unsigned long long p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Reads the device control block (synchronises the stream).
cc_status read_state(cc_ctx* c, DevState* out)
{
    CC_CUDA(c, cudaMemcpyAsync(out, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    return CC_OK;
}

cc_status read_jobs(cc_ctx* c, std::vector<JobState>& out)
{
    out.resize(c->jobs);
    CC_CUDA(c, cudaMemcpyAsync(out.data(), c->js, sizeof(JobState) * c->jobs, cudaMemcpyDeviceToHost, c->stream));
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    return CC_OK;
}

cc_status check_device_error(cc_ctx* c, const DevState& s)
{
    if (s.err == CC_ERR_TABLE_FULL) return fail(c, CC_ERR_TABLE_FULL, "contingency hash is full");
    if (s.err == CC_ERR_INVALID) return fail(c, CC_ERR_INVALID, "inconsistent contingency state");
    if (s.err != 0) return fail(c, (cc_status)s.err, "device-side failure");
    return CC_OK;
}

cc_status need_single(cc_ctx* c)
{
    if (c->jobs != 1) return fail(c, CC_ERR_INVALID, "this call needs a single-job context; use the cc_job_* calls");
    return CC_OK;
}

// F of every job recomputed from scratch (the table is built first if the
// context is still at the singleton start without one).
cc_status objective_recompute(cc_ctx* c, std::vector<long long>& F)
{
    DevState pre;
    cc_status rp = read_state(c, &pre);
    if (rp != CC_OK) return rp;
    if (!pre.tvalid) {
        CC_CUDA(c, cudaMemcpyAsync(&c->st->new_mask, &pre.mask, sizeof(pre.mask), cudaMemcpyHostToDevice, c->stream));
        CC_CUDA(c, launch_table_rebuild(c->args, c->rows, false, c->stream));
        c->launches += kKernelsPerRebuild;
    }
    CC_CUDA(c, launch_objective_recompute(c->args, c->stream));
    c->launches += 2;
    std::vector<JobState> js;
    cc_status r = read_jobs(c, js);
    if (r != CC_OK) return r;
    F.resize(c->jobs);
    for (int j = 0; j < c->jobs; ++j) F[j] = js[j].recompute + c->psq[j];
    DevState s;
    r = read_state(c, &s);
    if (r != CC_OK) return r;
    return check_device_error(c, s);
}

// Singleton start of every job: C[v] = v, sizes 1, F = F0, history cleared.
cc_status start_state(cc_ctx* c)
{
    DevState s;
    std::memset(&s, 0, sizeof(s));
    if (c->started) {
        DevState prev;
        cc_status rp = read_state(c, &prev);
        if (rp != CC_OK) return rp;
        s.rebuilds = prev.rebuilds;
        s.retries = prev.retries;
        s.region_launches = prev.region_launches;
    }
    c->started = true;
    s.stop = 1;
    s.cls = 0;
    s.ncls = c->ncls;
    s.new_mask = c->cap_start - 1;
    s.mask = c->cap_start - 1;
    std::vector<JobState> js(c->jobs);
    for (int j = 0; j < c->jobs; ++j) {
        std::memset(&js[j], 0, sizeof(JobState));
        js[j].F = c->F0[j];
        js[j].partition_sq = c->psq[j];
        js[j].stop = 1;
    }
    CC_CUDA(c, cudaMemcpyAsync(c->st, &s, sizeof(s), cudaMemcpyHostToDevice, c->stream));
    CC_CUDA(c, cudaMemcpyAsync(c->js, js.data(), sizeof(JobState) * c->jobs, cudaMemcpyHostToDevice, c->stream));
    CC_CUDA(c, launch_init_state(c->args, c->stream));
    if (c->opt.sweep_mode == 1) {
        // staged deltas need the singleton counts in the table from the start
        CC_CUDA(c, launch_table_rebuild(c->args, c->rows, false, c->stream));
        c->launches += 1 + kKernelsPerRebuild;
    } else {
        // the first sweep rebuilds the table itself (it is always heavy);
        // the summary rows of singletons follow from the label rows
        CC_CUDA(c, launch_singleton_summaries(c->args, c->rows, c->stream));
        c->launches += 2;
    }
    DevState r;
    cc_status rc = read_state(c, &r);
    if (rc != CC_OK) return rc;
    return check_device_error(c, r);
}

cc_status ensure_graph(cc_ctx* c, int limit, RunGraph** out)
{
    auto it = c->graphs.find(limit);
    if (it != c->graphs.end()) {
        *out = &it->second;
        return CC_OK;
    }
    RunGraph g;
    g.bound.resize((size_t)limit + 1);
    g.prop.resize(2 * (size_t)limit);
    for (auto& e : g.bound) CC_CUDA(c, cudaEventCreate(&e));
    for (auto& e : g.prop) CC_CUDA(c, cudaEventCreate(&e));
    cudaGraph_t graph = nullptr;
    CC_CUDA(c, cudaStreamBeginCapture(c->own_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < limit && e == cudaSuccess; ++s) {
        e = cudaEventRecordWithFlags(g.bound[s], c->own_stream, cudaEventRecordExternal);
        if (e == cudaSuccess)
            e = launch_sweep(c->args, c->rows, c->grid, c->own_stream, g.prop[2 * s], g.prop[2 * s + 1],
                             c->opt.no_regions ? nullptr : c->body_stream);
    }
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(g.bound[limit], c->own_stream, cudaEventRecordExternal);
    cudaStreamCaptureStatus bs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->body_stream, &bs) == cudaSuccess && bs != cudaStreamCaptureStatusNone) {
        cudaGraph_t body = nullptr;
        cudaStreamEndCapture(c->body_stream, &body);  // a region left open by a failed capture
    }
    cudaError_t e2 = cudaStreamEndCapture(c->own_stream, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        destroy_graph(g);
        return cuda_fail(c, e != cudaSuccess ? e : e2, "capture sweep graph");
    }
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        g.exec = nullptr;
        destroy_graph(g);
        return cuda_fail(c, e, "instantiate sweep graph");
    }
    auto ins = c->graphs.emplace(limit, g);
    *out = &ins.first->second;
    return CC_OK;
}

// A whole run of a multi-job context as one graph launch: a WHILE node
// repeats the sweep body until the run stops (at most `limit` sweeps' bodies
// plus 64 for abandoned and retried ones).  Returns the CUDA error instead of
// failing the context, so that the caller can fall back to chunks.
cudaError_t ensure_loop_graph(cc_ctx* c, int limit, RunGraph** out)
{
    auto it = c->graphs.find(-limit);
    if (it != c->graphs.end()) {
        *out = &it->second;
        return cudaSuccess;
    }
    RunGraph g;
    g.bound.resize(2);
    cudaError_t e = cudaSuccess;
    for (auto& ev : g.bound)
        if (e == cudaSuccess) e = cudaEventCreate(&ev);
    cudaGraph_t graph = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(c->own_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        e = cudaEventRecordWithFlags(g.bound[0], c->own_stream, cudaEventRecordExternal);
        const int budget = (int)std::min<long long>((long long)limit * c->ncls + 64, 1LL << 30);
        if (e == cudaSuccess)
            e = capture_run_loop(c->args, c->rows, c->grid, c->own_stream, c->loop_stream, c->body_stream, budget);
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(g.bound[1], c->own_stream, cudaEventRecordExternal);
        for (cudaStream_t st : {c->body_stream, c->loop_stream}) {
            cudaStreamCaptureStatus bs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(st, &bs) == cudaSuccess && bs != cudaStreamCaptureStatusNone) {
                cudaGraph_t left = nullptr;
                cudaStreamEndCapture(st, &left);  // a capture left open by a failure
                if (left) cudaGraphDestroy(left);
            }
        }
        const cudaError_t e2 = cudaStreamEndCapture(c->own_stream, &graph);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        g.exec = nullptr;
        destroy_graph(g);
        cudaGetLastError();  // the failure is reported to the caller, not left pending
        return e;
    }
    auto ins = c->graphs.emplace(-limit, g);
    *out = &ins.first->second;
    return cudaSuccess;
}

// Sweep bodies per graph launch: a run launches the graph until the device
// says the run has stopped, so at most kChunk - 1 skipped sweep bodies are
// submitted after the last sweep.  With colour_batched a body runs one colour
// class, and a graph holds up to kClassChunk of them.
constexpr int kChunk = 4;
constexpr int kClassChunk = 16;

int chunk_bodies(const cc_ctx* c, int limit)
{
    const long long bodies = (long long)limit * c->ncls;
    const int most = c->opt.colour_batched ? kClassChunk : kChunk;
    return bodies < most ? (int)bodies : most;
}

// Graph launches a run of `limit` sweeps may take: the bodies it needs plus
// 64 launches for sweeps abandoned for lack of table space and retried.
long long launch_budget(const cc_ctx* c, int limit, int chunk)
{
    return ((long long)limit * c->ncls + chunk - 1) / chunk + 64;
}

// Lane counts chosen by the autotuner, per device and lane bin (0 = none yet).
std::atomic<int> g_tuned[kMaxDevices][6];

int lane_bin(int k)
{
    int b = 0;
    for (int g = lanes_for_k(k); g > 1 && b < 5; g >>= 1) ++b;
    return b;
}

// Times the proposal kernels once per candidate lane count on the current
// state (each twice, the second kept) and keeps the fastest; the cached
// sweep graphs, which hold the old count, are dropped.
cc_status tune_lanes(cc_ctx* c)
{
    const int base = lanes_for_k(c->kmax);
    std::vector<int> cands;
    if (base > 1) cands.push_back(base / 2);
    cands.push_back(base);
    if (base < 32) cands.push_back(base * 2);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CC_CUDA(c, cudaEventCreate(&e0));
    CC_CUDA(c, cudaEventCreate(&e1));
    std::vector<float> ms(cands.size(), 0.f);
    cudaError_t e = cudaSuccess;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        for (size_t i = 0; i < cands.size() && e == cudaSuccess; ++i) {
            SweepArgs a = c->args;
            a.gs = cands[i];
            e = cudaEventRecord(e0, c->stream);
            if (e == cudaSuccess) e = launch_propose_probe(a, c->grid, c->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
            if (e == cudaSuccess) e = launch_clear_bids(a, c->grid, c->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[i], e0, e1);
            c->launches += 3;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(c, e, "autotune");
    size_t best = 0;
    for (size_t i = 1; i < cands.size(); ++i)
        if (ms[i] < ms[best]) best = i;
    c->args.gs = cands[best];
    for (auto& kv : c->graphs) destroy_graph(kv.second);
    c->graphs.clear();
    if (c->device >= 0 && c->device < kMaxDevices) g_tuned[c->device][lane_bin(c->kmax)].store(cands[best]);
    return CC_OK;
}

// Runs every job until it stops; *done = largest number of sweeps of a job in this run.
cc_status run(cc_ctx* c, int limit, int* done)
{
    const int full_limit = limit;
    CC_CUDA(c, launch_run_begin(c->args, limit, c->stream));
    c->launches += 1;
    c->sweep_ms.clear();
    c->propose_ms.clear();
    DevState st;
    int before = 0;
    cc_status r = CC_OK;
    if (!c->tuned) {
        // autotune: the run's first sweep alone, then the lane counts timed
        // on the state it left
        RunGraph* g1 = nullptr;
        r = ensure_graph(c, 1, &g1);
        if (r != CC_OK) return r;
        CC_CUDA(c, cudaGraphLaunch(g1->exec, c->stream));
        c->launches += c->opt.no_regions ? kKernelsPerSweep : kKernelsOutsideRegions;
        r = read_state(c, &st);
        if (r != CC_OK) return r;
        if (st.run_bodies > 0) {
            float x = 0.f, y = 0.f;
            CC_CUDA(c, cudaEventElapsedTime(&x, g1->bound[0], g1->bound[1]));
            CC_CUDA(c, cudaEventElapsedTime(&y, g1->prop[0], g1->prop[1]));
            c->sweep_ms.push_back(x);
            c->propose_ms.push_back(y);
        }
        before = st.run_bodies;
        if (!st.stop && !st.err) {
            r = tune_lanes(c);
            if (r != CC_OK) return r;
        }
        c->tuned = true;
        limit -= st.run_bodies > 0 ? 1 : 0;
    }
    // a multi-job context (unless profiling without regions) runs the rest as
    // one graph launch
    RunGraph* lg = nullptr;
    const bool loop = c->jobs > 1 && !c->opt.no_regions && c->loop_ok && !(before > 0 && (st.stop || st.err));
    if (loop && ensure_loop_graph(c, full_limit, &lg) != cudaSuccess) c->loop_ok = false;
    if (loop && c->loop_ok) {
        CC_CUDA(c, cudaGraphLaunch(lg->exec, c->stream));
        r = read_state(c, &st);
        if (r != CC_OK) return r;
        c->launches += (long long)(st.run_bodies - before) * (kKernelsOutsideRegions + 1);
        float x = 0.f;
        CC_CUDA(c, cudaEventElapsedTime(&x, lg->bound[0], lg->bound[1]));
        c->sweep_ms.push_back(x);
        c->propose_ms.push_back(0.f);
        before = st.run_bodies;
    }
    const int chunk = chunk_bodies(c, std::max(limit, 1));
    RunGraph* g = nullptr;
    if (!(before > 0 && (st.stop || st.err))) {
        r = ensure_graph(c, chunk, &g);
        if (r != CC_OK) return r;
    }
    // a sweep abandoned for lack of table space is retried in the next body,
    // so the number of launches is bounded by the limit plus the retries
    const long long budget = launch_budget(c, std::max(limit, 1), chunk);
    for (long long launch = 0; launch < budget && !(before > 0 && (st.stop || st.err)); ++launch) {
        CC_CUDA(c, cudaGraphLaunch(g->exec, c->stream));
        c->launches += (long long)chunk * (c->opt.no_regions ? kKernelsPerSweep : kKernelsOutsideRegions);
        r = read_state(c, &st);
        if (r != CC_OK) return r;
        const int ran = st.run_bodies - before;
        for (int b = 0; b < ran && b < chunk; ++b) {
            float x = 0.f, y = 0.f;
            CC_CUDA(c, cudaEventElapsedTime(&x, g->bound[b], g->bound[b + 1]));
            CC_CUDA(c, cudaEventElapsedTime(&y, g->prop[2 * b], g->prop[2 * b + 1]));
            c->sweep_ms.push_back(x);
            c->propose_ms.push_back(y);
        }
        before = st.run_bodies;
        if (st.stop || st.err) break;
    }
    r = check_device_error(c, st);
    if (r != CC_OK) return r;
    if (!st.stop) return fail(c, CC_ERR_TABLE_FULL, "sweep retries did not converge");
    std::vector<JobState> js;
    r = read_jobs(c, js);
    if (r != CC_OK) return r;
    int most = 0;
    for (const JobState& s : js) most = std::max(most, s.run_sweeps);
    if (done) *done = most;
    if (c->opt.debug_checks) {
        std::vector<long long> F;
        r = objective_recompute(c, F);
        if (r != CC_OK) return r;
        for (int j = 0; j < c->jobs; ++j)
            if (F[j] != js[j].F) return fail(c, CC_ERR_INVALID, "debug check: incremental objective differs from recomputed");
    }
    return CC_OK;
}

// Device bytes of one allocation of `bytes` (allocations are rounded up to
// 512 bytes or more).
inline size_t rounded(size_t bytes)
{
    return (std::max<size_t>(bytes, 16) + 511) & ~size_t(511);
}

}  // namespace

namespace ccg {

cc_options resolve_options(const cc_options* opt)
{
    cc_options o;
    if (opt) o = *opt;
    else cc_default_options(&o);
    if (o.max_sweeps <= 0) o.max_sweeps = 20;
    return o;
}

cc_status plan_jobs(int jobs, const JobInput* in, const cc_options& opt, Plan* out, std::string* msg)
{
    auto bad = [&](cc_status code, const std::string& m) {
        *msg = m;
        return code;
    };
    if (jobs < 1) return bad(CC_ERR_INVALID, "at least one job is needed");
    if (!in) return bad(CC_ERR_INVALID, "job descriptors are NULL");
    Plan p;
    p.jobs = jobs;
    for (int j = 0; j < jobs; ++j) {
        const JobInput& q = in[j];
        const std::string who = jobs > 1 ? "job " + std::to_string(j) + ": " : "";
        if (q.n < 1) return bad(CC_ERR_INVALID, who + "n must be >= 1");
        if (q.k < 1) return bad(CC_ERR_INVALID, who + "k must be >= 1");
        if (q.k > 4096) return bad(CC_ERR_INVALID, who + "k must be <= 4096");
        if (q.nnz < 0) return bad(CC_ERR_INVALID, who + "nnz must be >= 0");
        if (3LL * q.k * q.n + q.k >= (1LL << 31)) return bad(CC_ERR_OVERFLOW, who + "3 k n + k >= 2^31");
        p.n += q.n;
        p.nnz += q.nnz;
        p.rows += (long long)q.n * ((q.k + 3) & ~3);
        p.keys += (long long)q.n * q.k;
        p.parts += q.k;
        p.kmax = std::max(p.kmax, (int)q.k);
    }
    if (p.n >= (1LL << 31)) return bad(CC_ERR_OVERFLOW, "more than 2^31 - 1 vertices in all jobs together");
    if (opt.colour_batched && p.nnz >= (1LL << 31))
        return bad(CC_ERR_OVERFLOW, "colour_batched needs fewer than 2^31 CSR entries in all jobs together");
    cc_status r = check_options(opt, msg);
    if (r != CC_OK) return r;
    finish_plan(p, opt);
    *out = p;
    return CC_OK;
}

cc_status check_options(const cc_options& opt, std::string* msg)
{
    auto bad = [&](cc_status code, const std::string& m) {
        *msg = m;
        return code;
    };
    if (opt.no_regions != 0 && opt.no_regions != 1) return bad(CC_ERR_INVALID, "no_regions must be 0 or 1");
    if (opt.table_log2 < 0 || opt.table_log2 > 40) return bad(CC_ERR_INVALID, "table_log2 out of range");
    if (opt.table_start_log2 < 0 || opt.table_start_log2 > 40) return bad(CC_ERR_INVALID, "table_start_log2 out of range");
    if (opt.sweep_mode < 0 || opt.sweep_mode > 2) return bad(CC_ERR_INVALID, "sweep_mode must be 0, 1 or 2");
    if (opt.lanes < 0 || opt.lanes > 32 || (opt.lanes & (opt.lanes - 1)) != 0)
        return bad(CC_ERR_INVALID, "lanes must be 0 or a power of two up to 32");
    if (opt.active_set != 0 && opt.active_set != 1) return bad(CC_ERR_INVALID, "active_set must be 0 or 1");
    if (opt.empty_moves != 0 && opt.empty_moves != 1) return bad(CC_ERR_INVALID, "empty_moves must be 0 or 1");
    if (opt.colour_batched != 0 && opt.colour_batched != 1)
        return bad(CC_ERR_INVALID, "colour_batched must be 0 or 1");
    if (opt.colour_batched && opt.active_set) return bad(CC_ERR_INVALID, "colour_batched needs active_set = 0");
    if (opt.autotune != 0 && opt.autotune != 1) return bad(CC_ERR_INVALID, "autotune must be 0 or 1");
    if (opt.tight_rebuild < 0 || opt.tight_rebuild > 2) return bad(CC_ERR_INVALID, "tight_rebuild must be 0, 1 or 2");
    return CC_OK;
}

void finish_plan(Plan& p, const cc_options& opt)
{
    const int jobs = p.jobs;
    p.persistent = 0;
    p.temporary = 0;
    p.hist_cap = jobs == 1 ? (1 << 16) : std::max(64, (int)opt.max_sweeps);
    // a light sweep adds at most 2 x (the label rows its proposals move) keys,
    // at most 1/4 of sum k n when sweeps choose between light and heavy, so
    // 2 sum k n slots keep every sweep below the 7/8 fill limit; sweeps that
    // are always light may move every row and need twice that
    const unsigned long long want = (opt.sweep_mode == 1 ? 4ull : 2ull) * (unsigned long long)p.keys + 64;
    p.cap_max = opt.table_log2 > 0 ? (1ull << opt.table_log2) : next_pow2(want);
    if (p.cap_max < 64) p.cap_max = 64;
    p.cap_start = opt.table_start_log2 > 0 ? (1ull << opt.table_start_log2) : next_pow2(2ull * p.keys + 64);
    if (p.cap_start > p.cap_max) p.cap_start = p.cap_max;
    p.lcap = next_pow2(2ull * p.keys + 64);
    const size_t N = (size_t)p.n, J = (size_t)jobs;
    const size_t per[] = {
        sizeof(JobInfo) * (J + 1), sizeof(JobState) * (J + 1), 8 * (N + 1), 4 * (size_t)p.nnz, 4 * (size_t)p.nnz,
        4 * N, 4 * (size_t)p.rows, 16 * (size_t)p.rows, 4 * N, 4 * N, 4 * N, 8 * N, 4 * N,
        sizeof(Slot) * (size_t)p.cap_max, 4 * N, 4 * N, 4 * N, 4 * N, N, 4 * N, 4 * N, 4 * (N / 1024 + 2),
        4 * N, 8 * N, N, 4 * J, 8 * (J + 1), 8 * (size_t)p.parts, 8 * (size_t)p.parts,
        4 * (3 * N + N / 1024 + 64), sizeof(DevState), sizeof(cc_sweep_info) * J * (size_t)p.hist_cap};
    for (size_t b : per) p.persistent += rounded(b);
    if (opt.colour_batched) {
        // colour of each vertex, vertices and CSR entries listed by class,
        // class offsets (at most max degree + 1 classes, bounded by N + 1)
        const size_t cls[] = {4 * N, 4 * N, 4 * (size_t)p.nnz, 4 * (N + 2), 8 * (N + 2), 16 * (N + 2) + 8};
        for (size_t b : cls) p.persistent += rounded(b);
    }
    const size_t tmp[] = {8 * (N + J), 8 * (J + 1), 4 * (size_t)p.keys, 8 * (J + 1), 4 * (size_t)p.parts, 4 * J,
                          16 * (size_t)p.lcap};
    for (size_t b : tmp) p.temporary += rounded(b);
}

}  // namespace ccg

namespace {

cc_status create_common(int jobs, const JobInput* in, bool on_device, const cc_options* opt_in, void* stream,
                        cudaMemPool_t pool, cc_ctx** out, int priority = 0)
{
    if (!out) return fail(nullptr, CC_ERR_INVALID, "out is NULL");
    *out = nullptr;
    const cc_options opt = resolve_options(opt_in);
    Plan plan;
    std::string msg;
    cc_status pr = plan_jobs(jobs, in, opt, &plan, &msg);
    if (pr != CC_OK) return fail(nullptr, pr, msg);
    for (int j = 0; j < jobs; ++j)
        if (!in[j].row_off || !in[j].labels || (in[j].nnz > 0 && !in[j].col))
            return fail(nullptr, CC_ERR_INVALID, (jobs > 1 ? "job " + std::to_string(j) + ": " : std::string()) +
                                                     "null input pointer");
    const long long N = plan.n, NNZ = plan.nnz, rows = plan.rows, keys = plan.keys;
    const int kmax = plan.kmax;

    cc_ctx* c = new cc_ctx();
    c->jobs = jobs;
    c->kmax = kmax;
    c->n = N;
    c->nnz = NNZ;
    c->rows = rows;
    c->keys = keys;
    c->opt = opt;
    c->pool = pool;
    c->hist_cap = plan.hist_cap;

    auto bail = [&](cc_status code) {
        g_create_error = c->err;
        free_all(c);
        delete c;
        return code;
    };
#define CC_TRY(expr)                                                  \
    do {                                                              \
        cudaError_t e_ = (expr);                                      \
        if (e_ != cudaSuccess) return bail(cuda_fail(c, e_, #expr));  \
    } while (0)

    CC_TRY(cudaGetDevice(&c->device));
    CC_TRY(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device));
    CC_TRY(cudaStreamCreateWithPriority(&c->own_stream, cudaStreamNonBlocking, priority));
    CC_TRY(cudaStreamCreateWithPriority(&c->body_stream, cudaStreamNonBlocking, priority));
    CC_TRY(cudaStreamCreateWithPriority(&c->loop_stream, cudaStreamNonBlocking, priority));
    // pooled memory is allocated in the order of the context's own stream, so
    // such a context runs on that stream
    c->stream = (stream && !pool) ? static_cast<cudaStream_t>(stream) : c->own_stream;

    // job table
    c->job.resize(jobs);
    std::vector<long long> eo(jobs + 1, 0), lo(jobs + 1, 0);
    std::vector<int> pjob, pfirst(jobs);
    long long vo = 0, go = 0;
    for (int j = 0; j < jobs; ++j) {
        JobInfo& J = c->job[j];
        J.vo = vo;
        J.n = in[j].n;
        J.go = go;
        J.k = in[j].k;
        J.kp = (in[j].k + 3) & ~3;
        J.lshift = 0;
        while ((1LL << J.lshift) < J.n) ++J.lshift;
        J.pad = 0;
        vo += J.n;
        go += J.n * J.kp;
        eo[j + 1] = eo[j] + in[j].nnz;
        lo[j + 1] = lo[j] + (long long)in[j].k * in[j].n;
        pfirst[j] = (int)pjob.size();
        for (int i = 0; i < in[j].k; ++i) pjob.push_back(j);
    }
    c->pfirst = pfirst;
    c->eo = eo;
    c->slot_n.resize(jobs);
    c->slot_nnz.resize(jobs);
    c->slot_k.resize(jobs);
    for (int j = 0; j < jobs; ++j) {
        c->slot_n[j] = in[j].n;
        c->slot_nnz[j] = in[j].nnz;
        c->slot_k[j] = in[j].k;
    }
    c->parts = (int)pjob.size();
    c->lbase.assign(jobs + 1, 0);
    for (int j = 0; j < jobs; ++j) c->lbase[j + 1] = c->lbase[j] + ((long long)c->job[j].k << c->job[j].lshift);
    c->nlabels = c->lbase[jobs];

    const unsigned long long cap = plan.cap_max;
    c->cap_max = cap;

    CC_TRY(dalloc(c, &c->d_job, (size_t)jobs + 1));
    CC_TRY(dalloc(c, &c->d_pfirst, (size_t)jobs));
    CC_TRY(dalloc(c, &c->d_lbase, (size_t)jobs + 1));
    CC_TRY(dalloc(c, &c->part_sq, (size_t)plan.parts));
    CC_TRY(dalloc(c, &c->part_slog, (size_t)plan.parts));
    CC_TRY(dalloc(c, &c->js, (size_t)jobs + 1));
    CC_TRY(dalloc(c, &c->off, (size_t)N + 1));
    CC_TRY(dalloc(c, &c->col, (size_t)NNZ));
    CC_TRY(dalloc(c, &c->src, (size_t)NNZ));
    CC_TRY(dalloc(c, &c->jid, (size_t)N));
    CC_TRY(dalloc(c, &c->G, (size_t)rows));
    CC_TRY(dalloc(c, &c->summ, (size_t)rows));
    CC_TRY(dalloc(c, &c->C, (size_t)N));
    CC_TRY(dalloc(c, &c->size, (size_t)N));
    CC_TRY(dalloc(c, &c->dsize, (size_t)N));
    CC_TRY(dalloc(c, &c->best, (size_t)N));
    CC_TRY(dalloc(c, &c->aown, (size_t)N));
    CC_TRY(dalloc(c, &c->chg, (size_t)N));
    CC_TRY(dalloc(c, &c->prev, (size_t)N));
    CC_TRY(dalloc(c, &c->act, (size_t)N));
    CC_TRY(dalloc(c, &c->table, (size_t)cap));
    CC_TRY(dalloc(c, &c->pv, (size_t)N));
    CC_TRY(dalloc(c, &c->pa, (size_t)N));
    CC_TRY(dalloc(c, &c->pb, (size_t)N));
    CC_TRY(dalloc(c, &c->pg, (size_t)N));
    CC_TRY(dalloc(c, &c->pflag, (size_t)N));
    CC_TRY(dalloc(c, &c->members, (size_t)N));
    CC_TRY(dalloc(c, &c->cursor, (size_t)N));
    CC_TRY(dalloc(c, &c->bsum, (size_t)N / 1024 + 2));
    CC_TRY(dalloc(c, &c->scratch, 3 * (size_t)N + (size_t)N / 1024 + 64));
    CC_TRY(dalloc(c, &c->st, 1));
    CC_TRY(dalloc(c, &c->hist, (size_t)jobs * c->hist_cap));
    {
        // entry `jobs` is an idle job (no vertices, k = 0, always stopped) for
        // the vertices that a slot reloaded with a smaller job leaves unused
        std::vector<JobInfo> jt(c->job);
        jt.push_back(JobInfo{0, 0, 0, 0, 0, 0, 0});
        CC_TRY(cudaMemcpyAsync(c->d_job, jt.data(), sizeof(JobInfo) * ((size_t)jobs + 1), cudaMemcpyHostToDevice,
                               c->stream));
    }
    CC_TRY(cudaMemcpyAsync(c->d_lbase, c->lbase.data(), sizeof(long long) * (jobs + 1), cudaMemcpyHostToDevice,
                           c->stream));

    DevState s0;
    std::memset(&s0, 0, sizeof(s0));
    CC_TRY(cudaMemcpyAsync(c->st, &s0, sizeof(s0), cudaMemcpyHostToDevice, c->stream));
    std::vector<JobState> js0((size_t)jobs + 1);
    std::memset(js0.data(), 0, sizeof(JobState) * ((size_t)jobs + 1));
    js0[jobs].stop = 1;
    CC_TRY(cudaMemcpyAsync(c->js, js0.data(), sizeof(JobState) * ((size_t)jobs + 1), cudaMemcpyHostToDevice,
                           c->stream));
    js0.clear();

    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    // staging: offsets of every job whole (n + 1 each), labels partition-major per job
    {
        long long* offstage = nullptr;
        long long* d_eo = nullptr;
        int* labels = nullptr;
        long long* d_lo = nullptr;
        int* d_pjob = nullptr;
        void* lmap = nullptr;
        const unsigned long long lcap = plan.lcap;
        std::vector<void*> temp;
        auto tmalloc = [&](void** p, size_t bytes) {
            bytes = bytes > 0 ? bytes : 16;
            cudaError_t e = c->pool ? cudaMallocFromPoolAsync(p, bytes, c->pool, c->own_stream) : cudaMalloc(p, bytes);
            if (e == cudaSuccess) temp.push_back(*p);
            return e;
        };
        auto cleanup = [&]() {
            if (c->pool) {
                for (void* p : temp) cudaFreeAsync(p, c->own_stream);
            } else {
                cudaStreamSynchronize(c->stream);
                for (void* p : temp) cudaFree(p);
            }
        };
        cudaError_t e = tmalloc((void**)&offstage, sizeof(long long) * ((size_t)N + jobs));
        if (e == cudaSuccess) e = tmalloc((void**)&d_eo, sizeof(long long) * (jobs + 1));
        if (e == cudaSuccess) e = tmalloc((void**)&labels, sizeof(int) * (size_t)keys);
        if (e == cudaSuccess) e = tmalloc((void**)&d_lo, sizeof(long long) * (jobs + 1));
        if (e == cudaSuccess) e = tmalloc((void**)&d_pjob, sizeof(int) * pjob.size());
        int* d_pfirst = c->d_pfirst;
        if (e == cudaSuccess) e = tmalloc(&lmap, 16 * lcap);
        for (int j = 0; j < jobs && e == cudaSuccess; ++j) {
            const JobInfo& J = c->job[j];
            e = cudaMemcpyAsync(offstage + J.vo + j, in[j].row_off, sizeof(long long) * ((size_t)J.n + 1), kind, c->stream);
            if (e == cudaSuccess && in[j].nnz > 0)
                e = cudaMemcpyAsync(c->col + eo[j], in[j].col, sizeof(int) * (size_t)in[j].nnz, kind, c->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(labels + lo[j], in[j].labels, sizeof(int) * (size_t)(lo[j + 1] - lo[j]), kind, c->stream);
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_eo, eo.data(), sizeof(long long) * (jobs + 1), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_lo, lo.data(), sizeof(long long) * (jobs + 1), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_pjob, pjob.data(), sizeof(int) * pjob.size(), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_pfirst, pfirst.data(), sizeof(int) * jobs, cudaMemcpyHostToDevice, c->stream);
        AssemblyArgs as{};
        as.jobs = jobs;
        as.n = N;
        as.nnz = NNZ;
        as.offstage = offstage;
        as.eo = d_eo;
        as.job = c->d_job;
        as.off = c->off;
        as.col = c->col;
        as.src = c->src;
        as.jid = c->jid;
        as.st = c->st;
        if (e == cudaSuccess) e = launch_assemble(as, c->stream);
        DevState s;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&s, c->st, sizeof(s), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            cleanup();
            return bail(cuda_fail(c, e, "input assembly"));
        }
        if (s.err) {
            cleanup();
            return bail(fail(c, CC_ERR_INVALID, "malformed CSR: offsets must start at 0, end at nnz and not decrease; "
                                                "columns must lie in [0, n)"));
        }
        e = launch_assemble_edges(as, c->stream);
        LabelArgs la{};
        la.jobs = jobs;
        la.total = keys;
        la.labels = labels;
        la.lo = d_lo;
        la.pjob = d_pjob;
        la.pfirst = d_pfirst;
        la.job = c->d_job;
        la.js = c->js;
        la.G = c->G;
        la.lmap = lmap;
        la.lmask = lcap - 1;
        la.rows = rows;
        la.st = c->st;
        la.part_sq = c->part_sq;
        la.part_slog = c->part_slog;
        if (e == cudaSuccess) e = cudaMemsetAsync(c->part_sq, 0, sizeof(long long) * pjob.size(), c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->part_slog, 0, sizeof(double) * pjob.size(), c->stream);
        if (e == cudaSuccess) e = launch_compact_labels(la, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&s, c->st, sizeof(s), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        cleanup();
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "label compaction"));
        if (s.err) return bail(fail(c, CC_ERR_INVALID, "malformed CSR: columns must lie in [0, n)"));
    }
    std::vector<JobState> js;
    if (read_jobs(c, js) != CC_OK) return bail(CC_ERR_CUDA);
    c->F0.resize(jobs);
    c->psq.resize(jobs);
    for (int j = 0; j < jobs; ++j) {
        c->psq[j] = js[j].partition_sq;
        c->F0[j] = c->psq[j] - (long long)c->job[j].k * c->job[j].n;
    }
    c->cap_start = plan.cap_start;

    SweepArgs& a = c->args;
    a.n = N;
    a.nnz = NNZ;
    a.jobs = jobs;
    a.kmax = kmax;
    a.off = c->off;
    a.col = c->col;
    a.src = c->src;
    a.jid = c->jid;
    a.job = c->d_job;
    a.js = c->js;
    a.G = c->G;
    a.summ = c->summ;
    a.C = c->C;
    a.size = c->size;
    a.dsize = c->dsize;
    a.best = c->best;
    a.aown = c->aown;
    a.table = c->table;
    a.mask_max = cap - 1;
    a.cap_min = cap < 1024 ? cap : 1024;
    a.keys = (unsigned long long)keys;
    a.sweep_mode = c->opt.sweep_mode;
    a.gs = c->opt.lanes > 0 ? c->opt.lanes : lanes_for_k(kmax);
    // autotune: a choice made earlier on this device for the same lane bin is
    // used as it is; otherwise the first run times the candidates
    c->tuned = true;
    if (c->opt.autotune && c->opt.lanes == 0 && !c->opt.colour_batched) {
        int dev = 0;
        const int known = (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < kMaxDevices)
                              ? g_tuned[dev][lane_bin(kmax)].load()
                              : 0;
        if (known > 0) a.gs = known;
        else c->tuned = false;
    }
    a.active_set = c->opt.active_set;
    a.empty_moves = c->opt.empty_moves;
    a.tight_mode = c->opt.tight_rebuild;
    a.chg = c->chg;
    a.prev = c->prev;
    a.act = c->act;
    a.pv = c->pv;
    a.pa = c->pa;
    a.pb = c->pb;
    a.pg = c->pg;
    a.pflag = c->pflag;
    a.members = c->members;
    a.cursor = c->cursor;
    a.bsum = c->bsum;
    a.st = c->st;
    a.hist = c->hist;
    a.hist_cap = c->hist_cap;

    if (c->opt.colour_batched) {
        CC_TRY(dalloc(c, &c->colour, (size_t)N));
        CC_TRY(dalloc(c, &c->vlist, (size_t)N));
        CC_TRY(dalloc(c, &c->eidx, (size_t)NNZ));
        CC_TRY(dalloc(c, &c->voff, (size_t)N + 2));
        CC_TRY(dalloc(c, &c->eoff, (size_t)N + 2));
        CC_TRY(dalloc(c, &c->ccnt, 2 * ((size_t)N + 2) + 1));
        ColourArgs ca{};
        ca.n = N;
        ca.nnz = NNZ;
        ca.off = c->off;
        ca.col = c->col;
        ca.jid = c->jid;
        ca.job = c->d_job;
        ca.colour = c->colour;
        ca.vlist = c->vlist;
        ca.voff = c->voff;
        ca.eidx = c->eidx;
        ca.eoff = c->eoff;
        ca.cnt = c->ccnt;
        ca.flag = reinterpret_cast<int*>(c->ccnt + 2 * ((size_t)N + 2));
        int nc = 1;
        CC_TRY(launch_colouring(ca, &nc, c->stream));
        c->ncls = nc;
        a.colour_mode = 1;
        a.vlist = c->vlist;
        a.voff = c->voff;
        a.eidx = c->eidx;
        a.eoff = c->eoff;
    }

    int per_sm = 0;
    CC_TRY(prepare_propose(&per_sm));
    if (per_sm < 1) return bail(fail(c, CC_ERR_INVALID, "proposal kernel cannot be resident"));
    c->grid = c->sms * per_sm;

    cc_status rc = start_state(c);
    if (rc != CC_OK) return bail(rc);
    *out = c;
    return CC_OK;
#undef CC_TRY
}

// ---- output renumbering ----------------------------------------------------
// first[c] = least vertex of cluster c; flag[v] = 1 iff v is first of its
// cluster; rank = exclusive prefix sum of flags; label[v] = rank[first[C[v]]]
// minus rank[first vertex of v's job] (labels count from 0 in each job).
__global__ void k_first(long long n, int* first)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) first[v] = 0x7fffffff;
}

__global__ void k_first_min(long long n, const int* __restrict__ C, int* first)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) atomicMin(&first[C[v]], (int)v);
}

__global__ void k_flags(long long n, const int* __restrict__ C, const int* __restrict__ first, int* flag, int* blocksum)
{
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int f = 0;
    if (v < n) f = first[C[v]] == v;
    if (v < n) flag[v] = f;
    if (f) atomicAdd(&cnt, 1);
    __syncthreads();
    if (threadIdx.x == 0) blocksum[blockIdx.x] = cnt;
}

// Exclusive scan of the nb block counts by one block of 1024 threads, each
// owning a contiguous run of counts.
__global__ void k_scan_counts(int nb, int* blocksum)
{
    __shared__ int part[1024];
    const int per = (nb + 1023) / 1024;
    const int lo = threadIdx.x * per, hi = min(nb, lo + per);
    int sum = 0;
    for (int b = lo; b < hi; ++b) sum += blocksum[b];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int y = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += y;
        __syncthreads();
    }
    int run = part[threadIdx.x] - sum;
    for (int b = lo; b < hi; ++b) {
        const int x = blocksum[b];
        blocksum[b] = run;
        run += x;
    }
}

// Within-block exclusive scan of the flags plus the block offset -> rank in place.
__global__ void k_rank(long long n, int* flag, const int* blocksum)
{
    __shared__ int buf[1024];
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int f = v < n ? flag[v] : 0;
    buf[threadIdx.x] = f;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        int y = threadIdx.x >= (unsigned)o ? buf[threadIdx.x - o] : 0;
        __syncthreads();
        buf[threadIdx.x] += y;
        __syncthreads();
    }
    if (v < n) flag[v] = blocksum[blockIdx.x] + buf[threadIdx.x] - f;
}

__global__ void k_relabel(long long n, const int* __restrict__ C, const int* __restrict__ first,
                          const int* __restrict__ rank, const int* __restrict__ jid, const JobInfo* __restrict__ job,
                          int* out)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        out[v] = rank[first[C[v]]] - rank[job[jid[v]].vo];
}

// Job-local cluster ids (C[v] - first vertex of v's job), or the reverse.
__global__ void k_shift_ids(long long n, const int* __restrict__ in, const int* __restrict__ jid,
                            const JobInfo* __restrict__ job, int sign, int* out)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        out[v] = (int)((unsigned)in[v] + (unsigned)sign * (unsigned)job[jid[v]].vo);
}

// ---- loading a job into a finished job's place (served form) -------------

// The new job's CSR: offsets start at 0, do not decrease, end at nnz;
// columns lie in [0, n).
__global__ void k_load_check(long long n, long long nnz, const long long* __restrict__ ro,
                             const int* __restrict__ col, DevState* st)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long t = t0; t < n; t += stride)
        if (ro[t + 1] < ro[t]) atomicCAS(&st->err, 0, (int)CC_ERR_INVALID);
    for (long long e = t0; e < nnz; e += stride)
        if (col[e] < 0 || col[e] >= n) atomicCAS(&st->err, 0, (int)CC_ERR_INVALID);
    if (t0 == 0 && (ro[0] != 0 || ro[n] != nnz)) atomicCAS(&st->err, 0, (int)CC_ERR_INVALID);
}

// Place of ncap vertices from vo and nnzcap CSR entries from eo: vertex t < n
// gets row ro[t] .. ro[t + 1], the last one also the unused entries (as
// self-loops); vertices t >= n get empty rows and the idle job.
__global__ void k_load_csr(long long vo, long long n, long long ncap, long long eo, long long nnz, long long nnzcap,
                           const long long* __restrict__ ro, const int* __restrict__ col_in, int job, int idle,
                           long long* off, int* col, int* jid)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long t = t0; t < ncap; t += stride) {
        off[vo + t] = eo + (t < n ? ro[t] : nnzcap);
        jid[vo + t] = t < n ? job : idle;
    }
    for (long long e = t0; e < nnzcap; e += stride)
        col[eo + e] = (int)(vo + (e < nnz ? col_in[e] : n - 1));
}

// Source vertex of every CSR entry of the place, one thread per entry: the
// vertex whose row holds it (binary search in the new job's offsets; the
// unused entries at the end belong to its last vertex).
__global__ void k_load_src(long long vo, long long n, long long eo, long long nnz, long long nnzcap,
                           const long long* __restrict__ ro, int* src)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nnzcap; e += stride) {
        long long v = n - 1;
        if (e < nnz) {
            long long lo = 0, hi = n - 1;  // last t with ro[t] <= e
            while (lo < hi) {
                const long long mid = (lo + hi + 1) >> 1;
                if (ro[mid] <= e) lo = mid;
                else hi = mid - 1;
            }
            v = lo;
        }
        src[eo + e] = (int)(vo + v);
    }
}

// The finished job's contingency keys (its clusters' ids lie in its place)
// get count 0 before its state is overwritten; the table stays valid for the
// other jobs.  Skipped if the table does not hold the counts of C.
__global__ void k_unload_keys(SweepArgs a, JobInfo J, long long vo)
{
    if (!a.st->tvalid) return;
    const unsigned long long mask = a.st->mask;
    const long long total = J.n * J.k, stride = (long long)gridDim.x * blockDim.x;
    long long dead = 0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const long long vl = t / J.k;
        const int i = (int)(t - vl * J.k);
        const int g = a.G[J.go + vl * J.kp + i];
        const long long s = table_find(a.table, mask, ckey(a.C[vo + vl], g));
        if (s >= 0 && atomicExch(&a.table[s].cnt, 0) > 0) ++dead;
    }
    if (dead) atomicAdd(reinterpret_cast<unsigned long long*>(&a.st->live), (unsigned long long)(-dead));
}

// The new job's singleton keys, count 1 each.  If the table runs short, it is
// marked as not holding the counts, so that the next sweep rebuilds it.
__global__ void k_load_keys(SweepArgs a, JobInfo J, long long vo)
{
    DevState* st = a.st;
    if (!st->tvalid) return;
    const unsigned long long mask = st->mask;
    const long long total = J.n * J.k, stride = (long long)gridDim.x * blockDim.x;
    long long live = 0, used = 0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const long long vl = t / J.k;
        const int i = (int)(t - vl * J.k);
        bool ins = false;
        const long long s = table_find_or_insert(a.table, mask, ckey((int)(vo + vl), a.G[J.go + vl * J.kp + i]), &ins);
        if (s < 0) {
            st->tvalid = 0;
            continue;
        }
        used += ins ? 1 : 0;
        if (atomicAdd(&a.table[s].cnt, 1) == 0) ++live;
    }
    if (live) atomicAdd(reinterpret_cast<unsigned long long*>(&st->live), (unsigned long long)live);
    if (used) atomicAdd(&st->used, (unsigned long long)used);
}

// Before the new job's keys go in: if they could take the table past 7/8
// of its slots (the finished job's keys still hold theirs), they are not
// inserted and the next sweep rebuilds the table from C instead, so that
// probing never runs in a nearly full table.
__global__ void k_load_check_fill(DevState* st, unsigned long long new_keys)
{
    const unsigned long long cap = st->mask + 1;
    if (st->used + new_keys > cap - (cap >> 3)) st->tvalid = 0;
}

// Singleton state of the place's vertices (stamped as changed in the sweep
// just run, so that the next sweep computes their own-cluster sums) and the
// summary rows of the new job's label rows; the run goes on.
__global__ void k_load_state(SweepArgs a, long long vo, long long ncap, long long go, long long rows)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int stamp = a.st->stamp;
    for (long long t = t0; t < ncap; t += stride) {
        const long long v = vo + t;
        a.C[v] = (int)v;
        a.size[v] = 1;
        a.dsize[v] = 0;
        a.best[v] = kEmpty;
        a.chg[v] = stamp;
        a.prev[v] = kEmpty;
        a.act[v] = 1;
    }
    for (long long r = t0; r < rows; r += stride) {
        const int g = a.G[go + r];
        a.summ[go + r] = make_int4(g, g >= 0 ? 1 : 0, -1, 0);
    }
    if (t0 == 0) a.st->stop = 0;
}

// Job-local renumbering of one job (vertices vo .. vo + n - 1): first holds,
// at each of the job's cluster ids, the least job-local index of its members.
__global__ void k_first_min_job(long long n, long long vo, const int* __restrict__ C, int* first)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride)
        atomicMin(&first[C[vo + t]], (int)t);
}

__global__ void k_flags_job(long long n, long long vo, const int* __restrict__ C, const int* __restrict__ first,
                            int* flag, int* blocksum)
{
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int f = 0;
    if (t < n) f = first[C[vo + t]] == t;
    if (t < n) flag[t] = f;
    if (f) atomicAdd(&cnt, 1);
    __syncthreads();
    if (threadIdx.x == 0) blocksum[blockIdx.x] = cnt;
}

__global__ void k_relabel_job(long long n, long long vo, const int* __restrict__ C, const int* __restrict__ first,
                              const int* __restrict__ rank, int* out)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride)
        out[t] = rank[first[C[vo + t]]];
}

// Renumbered labels of job j alone into scratch + 2N + vo_j (device); the
// scratch ranges of other jobs are not touched.
cc_status renumber_job(cc_ctx* c, int j, int** labels)
{
    const long long N = c->n, vo = c->job[j].vo, n = c->job[j].n;
    int* first = c->scratch;                 // indexed by (union) cluster id: the job's ids
    int* rank = c->scratch + N + vo;         // job-local
    int* lab = c->scratch + 2 * (size_t)N + vo;
    int* blocksum = c->scratch + 3 * (size_t)N;
    const int nb = (int)((n + 1023) / 1024);
    const int g = std::max(1, std::min(c->sms * 8, (int)((n + 255) / 256)));
    k_first<<<g, 256, 0, c->stream>>>(n, first + vo);
    k_first_min_job<<<g, 256, 0, c->stream>>>(n, vo, c->C, first);
    k_flags_job<<<nb, 1024, 0, c->stream>>>(n, vo, c->C, first, rank, blocksum);
    k_scan_counts<<<1, 1024, 0, c->stream>>>(nb, blocksum);
    k_rank<<<nb, 1024, 0, c->stream>>>(n, rank, blocksum);
    k_relabel_job<<<g, 256, 0, c->stream>>>(n, vo, c->C, first, rank, lab);
    c->launches += 6;
    CC_CUDA(c, cudaGetLastError());
    *labels = lab;
    return CC_OK;
}

// Renumbered labels of every vertex into scratch + 2n (device); returns that pointer.
cc_status renumber(cc_ctx* c, int** labels)
{
    const long long n = c->n;
    int* first = c->scratch;
    int* rank = c->scratch + n;
    int* lab = c->scratch + 2 * (size_t)n;
    int* blocksum = c->scratch + 3 * (size_t)n;
    const int nb = (int)((n + 1023) / 1024);
    const int g = c->sms * 8;
    k_first<<<g, 256, 0, c->stream>>>(n, first);
    k_first_min<<<g, 256, 0, c->stream>>>(n, c->C, first);
    k_flags<<<nb, 1024, 0, c->stream>>>(n, c->C, first, rank, blocksum);
    k_scan_counts<<<1, 1024, 0, c->stream>>>(nb, blocksum);
    k_rank<<<nb, 1024, 0, c->stream>>>(n, rank, blocksum);
    k_relabel<<<g, 256, 0, c->stream>>>(n, c->C, first, rank, c->jid, c->d_job, lab);
    c->launches += 6;
    CC_CUDA(c, cudaGetLastError());
    *labels = lab;
    return CC_OK;
}

cc_status check_job(cc_ctx* c, int32_t job)
{
    if (!c) return fail(nullptr, CC_ERR_INVALID, "ctx is NULL");
    if (job < 0 || job >= c->jobs) return fail(c, CC_ERR_INVALID, "job index out of range");
    return CC_OK;
}

cc_status launch_chunk(cc_ctx* c)
{
    const int chunk = chunk_bodies(c, c->async_limit);
    RunGraph* g = nullptr;
    cc_status r = ensure_graph(c, chunk, &g);
    if (r != CC_OK) return r;
    CC_CUDA(c, cudaGraphLaunch(g->exec, c->stream));
    c->launches += (long long)chunk * (c->opt.no_regions ? kKernelsPerSweep : kKernelsOutsideRegions);
    CC_CUDA(c, cudaMemcpyAsync(c->hstate, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    if (c->hjobs)
        CC_CUDA(c, cudaMemcpyAsync(c->hjobs, c->js, sizeof(JobState) * (size_t)c->jobs, cudaMemcpyDeviceToHost,
                                   c->stream));
    CC_CUDA(c, cudaEventRecord(c->chunk_done, c->stream));
    c->async_launches += 1;
    return CC_OK;
}

}  // namespace

namespace ccg {

cc_status ctx_create(int jobs, const JobInput* in, bool on_device, const cc_options* opt, void* stream,
                     cudaMemPool_t pool, cc_ctx** out, int priority)
{
    return create_common(jobs, in, on_device, opt, stream, pool, out, priority);
}

cc_status ctx_async_start(cc_ctx* c, int limit, DevState* pinned, JobState* pinned_jobs)
{
    c->hstate = pinned;
    c->hjobs = pinned_jobs;
    c->async_limit = limit > 0 ? limit : c->opt.max_sweeps;
    c->async_launches = 0;
    if (!c->chunk_done) CC_CUDA(c, cudaEventCreateWithFlags(&c->chunk_done, cudaEventDisableTiming));
    CC_CUDA(c, launch_run_begin(c->args, c->async_limit, c->stream));
    c->launches += 1;
    return launch_chunk(c);
}

int ctx_async_poll(cc_ctx* c, cc_status* st)
{
    const int r = ctx_async_poll_step(c, st);
    if (r != 2) return r;
    *st = ctx_async_continue(c);
    return *st == CC_OK ? 0 : -1;
}

cc_status ctx_async_continue(cc_ctx* c)
{
    return launch_chunk(c);
}

int ctx_async_poll_step(cc_ctx* c, cc_status* st)
{
    *st = CC_OK;
    const cudaError_t q = cudaEventQuery(c->chunk_done);
    if (q == cudaErrorNotReady) return 0;
    if (q != cudaSuccess) {
        *st = cuda_fail(c, q, "sweep chunk");
        return -1;
    }
    const DevState s = *c->hstate;
    if (s.err) {
        *st = check_device_error(c, s);
        return -1;
    }
    if (s.stop) return 1;
    // each launch runs up to chunk_bodies sweep bodies; abandoned sweeps are retried
    if (c->async_launches > launch_budget(c, c->async_limit, chunk_bodies(c, c->async_limit))) {
        *st = fail(c, CC_ERR_TABLE_FULL, "sweep retries did not converge");
        return -1;
    }
    return 2;
}

cc_status ctx_job_results(cc_ctx* c, std::vector<long long>& F, std::vector<int>& sweeps)
{
    std::vector<JobState> js;
    cc_status r = read_jobs(c, js);
    if (r != CC_OK) return r;
    F.resize(c->jobs);
    sweeps.resize(c->jobs);
    for (int j = 0; j < c->jobs; ++j) {
        F[j] = js[j].F;
        sweeps[j] = js[j].sweeps;
    }
    return CC_OK;
}

cc_status ctx_renumber(cc_ctx* c, int** dev_labels)
{
    return renumber(c, dev_labels);
}

cc_status ctx_copy_labels(cc_ctx* c, const int* dev_labels, int j, int32_t* out)
{
    const JobInfo& J = c->job[j];
    CC_CUDA(c, cudaMemcpyAsync(out, dev_labels + J.vo, sizeof(int) * (size_t)J.n, cudaMemcpyDeviceToHost, c->stream));
    return CC_OK;
}

bool ctx_slot_fits(const cc_ctx* c, int j, const JobInput& in)
{
    const long long kp_new = (in.k + 3) & ~3, kp_cap = (c->slot_k[j] + 3) & ~3;
    // no larger than the place, and not much smaller: every sweep scans the
    // whole place, so a small job in a large place would pay for it
    return !c->opt.colour_batched && in.n >= 1 && in.n <= c->slot_n[j] && in.nnz <= c->slot_nnz[j] &&
           4LL * in.n >= c->slot_n[j] && 4LL * in.nnz >= c->slot_nnz[j] && in.k >= 1 && in.k <= c->slot_k[j] &&
           (long long)in.n * kp_new <= c->slot_n[j] * kp_cap &&
           (long long)in.n * in.k <= c->slot_n[j] * (long long)c->slot_k[j] && in.k <= c->kmax;
}

cc_status ctx_load_job(cc_ctx* c, int j, const JobInput& in)
{
    if (j < 0 || j >= c->jobs || !ctx_slot_fits(c, j, in) || !in.row_off || !in.labels || (in.nnz > 0 && !in.col))
        return fail(c, CC_ERR_INVALID, "job does not fit the place it is loaded into");
    const long long n = in.n, nnz = in.nnz, k = in.k;
    const long long ncap = c->slot_n[j], nnzcap = c->slot_nnz[j];
    JobInfo J = c->job[j];
    J.n = n;
    J.k = (int)k;
    J.kp = (int)((k + 3) & ~3);
    J.lshift = 0;
    while ((1LL << J.lshift) < n) ++J.lshift;
    const long long eo = c->eo[j], keys = n * k;
    unsigned long long lcap = 64;
    while (lcap < 2ull * (unsigned long long)keys + 64) lcap <<= 1;
    // staging, from the context's pool when it has one (stream-ordered)
    std::vector<void*> temp;
    auto tmalloc = [&](void** p, size_t bytes) {
        bytes = bytes > 0 ? bytes : 16;
        cudaError_t e = c->pool ? cudaMallocFromPoolAsync(p, bytes, c->pool, c->stream) : cudaMalloc(p, bytes);
        if (e == cudaSuccess) temp.push_back(*p);
        return e;
    };
    auto cleanup = [&]() {
        if (c->pool) {
            for (void* p : temp) cudaFreeAsync(p, c->stream);
        } else {
            cudaStreamSynchronize(c->stream);
            for (void* p : temp) cudaFree(p);
        }
    };
    long long *ro = nullptr, *lo = nullptr;
    int *col = nullptr, *lab = nullptr, *pjob = nullptr, *pfirst = nullptr;
    void* lmap = nullptr;
    JobInfo* dj = nullptr;
    DevState* tst = nullptr;
    cudaError_t e = tmalloc((void**)&ro, sizeof(long long) * ((size_t)n + 1));
    if (e == cudaSuccess) e = tmalloc((void**)&col, sizeof(int) * (size_t)nnz);
    if (e == cudaSuccess) e = tmalloc((void**)&lab, sizeof(int) * (size_t)keys);
    if (e == cudaSuccess) e = tmalloc((void**)&lo, sizeof(long long) * 2);
    if (e == cudaSuccess) e = tmalloc((void**)&pjob, sizeof(int) * (size_t)k);
    if (e == cudaSuccess) e = tmalloc((void**)&pfirst, sizeof(int));
    if (e == cudaSuccess) e = tmalloc(&lmap, 16 * (size_t)lcap);
    if (e == cudaSuccess) e = tmalloc((void**)&dj, sizeof(JobInfo));
    if (e == cudaSuccess) e = tmalloc((void**)&tst, sizeof(DevState));
    const long long lo_h[2] = {0, keys};
    const int zero = 0;
    DevState s0;
    std::memset(&s0, 0, sizeof(s0));
    if (e == cudaSuccess) e = cudaMemcpyAsync(ro, in.row_off, sizeof(long long) * ((size_t)n + 1), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(col, in.col, sizeof(int) * (size_t)nnz, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(lab, in.labels, sizeof(int) * (size_t)keys, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(lo, lo_h, sizeof(lo_h), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(pjob, 0, sizeof(int) * (size_t)k, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pfirst, &zero, sizeof(int), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dj, &J, sizeof(JobInfo), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tst, &s0, sizeof(DevState), cudaMemcpyHostToDevice, c->stream);
    const int g = std::max(1, std::min(c->sms * 8, (int)((std::max(ncap, nnzcap) + 255) / 256)));
    // check the new job's CSR before anything of the context changes
    if (e == cudaSuccess) {
        k_load_check<<<g, 256, 0, c->stream>>>(n, nnz, ro, col, tst);
        e = cudaGetLastError();
    }
    DevState chk;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&chk, tst, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(c, e, "load job: staging");
    }
    if (chk.err) {
        cleanup();
        return fail(c, CC_ERR_INVALID, "malformed CSR: offsets must start at 0, end at nnz and not decrease; "
                                       "columns must lie in [0, n)");
    }
    // the finished job's keys leave the table
    k_unload_keys<<<g, 256, 0, c->stream>>>(c->args, c->job[j], J.vo);
    // the graph into the place: offsets, columns (union ids; unused entries
    // become self-loops of the last vertex), job of each vertex, sources
    k_load_csr<<<g, 256, 0, c->stream>>>(J.vo, n, ncap, eo, nnz, nnzcap, ro, col, j, c->jobs, c->off, c->col, c->jid);
    k_load_src<<<g, 256, 0, c->stream>>>(J.vo, n, eo, nnz, nnzcap, ro, c->src);
    // labels: compacted as at creation, into the place's rows
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(c->G + J.go, 0xff, sizeof(int) * (size_t)(n * J.kp), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->part_sq + c->pfirst[j], 0, sizeof(long long) * (size_t)k, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->part_slog + c->pfirst[j], 0, sizeof(double) * (size_t)k, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&c->js[j], 0, sizeof(JobState), c->stream);
    LabelArgs la{};
    la.jobs = 1;
    la.total = keys;
    la.labels = lab;
    la.lo = lo;
    la.pjob = pjob;
    la.pfirst = pfirst;
    la.job = dj;
    la.js = c->js + j;
    la.G = c->G;
    la.lmap = lmap;
    la.lmask = lcap - 1;
    la.rows = n * J.kp;
    la.st = tst;
    la.part_sq = c->part_sq + c->pfirst[j];
    la.part_slog = c->part_slog + c->pfirst[j];
    if (e == cudaSuccess) e = launch_label_kernels(la, c->stream);
    // singleton state of the place's vertices, their summary rows, and a
    // table rebuild in the next sweep
    if (e == cudaSuccess) {
        k_load_state<<<g, 256, 0, c->stream>>>(c->args, J.vo, ncap, J.go, n * J.kp);
        k_load_check_fill<<<1, 1, 0, c->stream>>>(c->st, (unsigned long long)keys);
        k_load_keys<<<g, 256, 0, c->stream>>>(c->args, J, J.vo);
        e = cudaGetLastError();
    }
    JobState jsr;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&jsr, &c->js[j], sizeof(JobState), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&chk, tst, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(c, e, "load job");
    }
    if (chk.err) {
        cleanup();
        return fail(c, CC_ERR_CUDA, "load job: label compaction failed");
    }
    const long long psq = jsr.partition_sq;
    std::memset(&jsr, 0, sizeof(jsr));
    jsr.partition_sq = psq;
    jsr.F = psq - k * n;
    e = cudaMemcpyAsync(&c->js[j], &jsr, sizeof(JobState), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_job + j, &J, sizeof(JobInfo), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // jsr and J are host locals
    cleanup();
    if (e != cudaSuccess) return cuda_fail(c, e, "load job: records");
    c->job[j] = J;
    c->psq[j] = psq;
    c->F0[j] = psq - k * n;
    c->async_launches = 0;  // the run's launch budget starts again
    return CC_OK;
}

cc_status ctx_job_labels_now(cc_ctx* c, int j, int32_t* out)
{
    int* lab = nullptr;
    cc_status r = renumber_job(c, j, &lab);
    if (r != CC_OK) return r;
    CC_CUDA(c, cudaMemcpyAsync(out, lab, sizeof(int) * (size_t)c->job[j].n, cudaMemcpyDeviceToHost, c->stream));
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    return CC_OK;
}

void ctx_destroy(cc_ctx* c)
{
    if (!c) return;
    if (!c->pool && c->stream) cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

}  // namespace ccg

extern "C" {

cc_status cc_estimate_bytes(int32_t jobs, const cc_job_desc* descs, const cc_options* opt, int64_t* persistent,
                            int64_t* peak)
{
    if (jobs < 1 || !descs) return fail(nullptr, CC_ERR_INVALID, "cc_estimate_bytes needs jobs >= 1 and descriptors");
    std::vector<JobInput> in(jobs);
    for (int j = 0; j < jobs; ++j)
        in[j] = JobInput{descs[j].n, descs[j].nnz, descs[j].row_off, descs[j].col, descs[j].k, descs[j].labels};
    Plan p;
    std::string msg;
    cc_status r = plan_jobs(jobs, in.data(), resolve_options(opt), &p, &msg);
    if (r != CC_OK) return fail(nullptr, r, msg);
    if (persistent) *persistent = (int64_t)p.persistent;
    if (peak) *peak = (int64_t)(p.persistent + p.temporary);
    return CC_OK;
}


void cc_default_options(cc_options* opt)
{
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->max_sweeps = 20;
}

cc_status cc_autotune_record(int32_t bins, int32_t* out)
{
    if (!out) return fail(nullptr, CC_ERR_INVALID, "out is NULL");
    int dev = 0;
    const bool ok = cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < kMaxDevices;
    for (int b = 0; b < bins && b < 6; ++b) out[b] = ok ? g_tuned[dev][b].load() : 0;
    return CC_OK;
}

cc_status cc_create(int32_t n, int64_t nnz, const int64_t* row_off, const int32_t* col, int32_t k,
                    const int32_t* labels, const cc_options* opt, cc_ctx** out)
{
    const JobInput in{n, nnz, row_off, col, k, labels};
    return create_common(1, &in, false, opt, nullptr, nullptr, out);
}

cc_status cc_create_dev(int32_t n, int64_t nnz, const int64_t* row_off_dev, const int32_t* col_dev, int32_t k,
                        const int32_t* labels_dev, const cc_options* opt, void* stream, cc_ctx** out)
{
    const JobInput in{n, nnz, row_off_dev, col_dev, k, labels_dev};
    return create_common(1, &in, true, opt, stream, nullptr, out);
}

cc_status cc_batch_create(int32_t jobs, const cc_job_desc* descs, const cc_options* opt, cc_ctx** out)
{
    if (jobs < 1 || !descs) {
        if (out) *out = nullptr;
        return fail(nullptr, CC_ERR_INVALID, "cc_batch_create needs jobs >= 1 and descriptors");
    }
    std::vector<JobInput> in(jobs);
    for (int j = 0; j < jobs; ++j)
        in[j] = JobInput{descs[j].n, descs[j].nnz, descs[j].row_off, descs[j].col, descs[j].k, descs[j].labels};
    return create_common(jobs, in.data(), false, opt, nullptr, nullptr, out);
}

cc_status cc_set_stream(cc_ctx* c, void* stream)
{
    if (!c) return fail(nullptr, CC_ERR_INVALID, "ctx is NULL");
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    c->stream = stream ? static_cast<cudaStream_t>(stream) : c->own_stream;
    return CC_OK;
}

cc_status cc_reset(cc_ctx* c)
{
    if (!c) return fail(nullptr, CC_ERR_INVALID, "ctx is NULL");
    return start_state(c);
}

cc_status cc_set_cluster_ids(cc_ctx* c, const int32_t* C)
{
    if (!c || !C) return fail(c, CC_ERR_INVALID, "null argument");
    const long long n = c->n;
    // job-local ids -> union ids in scratch[n .. 2n), checked before C is touched
    CC_CUDA(c, cudaMemcpyAsync(c->scratch, C, sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, c->stream));
    k_shift_ids<<<c->sms * 8, 256, 0, c->stream>>>(n, c->scratch, c->jid, c->d_job, 1, c->scratch + n);
    DevState s;
    cc_status r = read_state(c, &s);
    if (r != CC_OK) return r;
    CC_CUDA(c, cudaMemsetAsync(&c->st->err, 0, sizeof(int), c->stream));
    SweepArgs probe = c->args;
    probe.C = c->scratch + n;
    probe.size = c->scratch;  // the job-local copy is no longer needed
    probe.dsize = c->scratch + 2 * (size_t)n;
    probe.best = c->best;
    CC_CUDA(c, launch_state_from_ids(probe, c->stream));
    c->launches += 3;
    DevState chk;
    r = read_state(c, &chk);
    if (r != CC_OK) return r;
    if (chk.err) {
        CC_CUDA(c, cudaMemcpyAsync(&c->st->err, &s.err, sizeof(int), cudaMemcpyHostToDevice, c->stream));
        CC_CUDA(c, cudaStreamSynchronize(c->stream));
        return fail(c, CC_ERR_INVALID, "cluster ids must lie in [0, n) of their job");
    }
    CC_CUDA(c, cudaMemcpyAsync(c->C, c->scratch + n, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, c->stream));
    const unsigned long long nm = c->cap_start - 1;
    CC_CUDA(c, cudaMemcpyAsync(&c->st->new_mask, &nm, sizeof(nm), cudaMemcpyHostToDevice, c->stream));
    CC_CUDA(c, launch_state_from_ids(c->args, c->stream));
    CC_CUDA(c, launch_table_rebuild(c->args, c->rows, false, c->stream));
    c->launches += 2 + kKernelsPerRebuild;
    std::vector<long long> F;
    r = objective_recompute(c, F);
    if (r != CC_OK) return r;
    std::vector<JobState> js;
    r = read_jobs(c, js);
    if (r != CC_OK) return r;
    for (int j = 0; j < c->jobs; ++j) {
        js[j].F = F[j];
        js[j].stop = 1;
    }
    CC_CUDA(c, cudaMemcpyAsync(c->js, js.data(), sizeof(JobState) * c->jobs, cudaMemcpyHostToDevice, c->stream));
    int one = 1;
    CC_CUDA(c, cudaMemcpyAsync(&c->st->stop, &one, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    DevState after;
    r = read_state(c, &after);
    if (r != CC_OK) return r;
    return check_device_error(c, after);
}

cc_status cc_job_history(cc_ctx* c, int32_t job, int32_t max, cc_sweep_info* out, int32_t* count)
{
    cc_status r = check_job(c, job);
    if (r != CC_OK) return r;
    std::vector<JobState> js;
    r = read_jobs(c, js);
    if (r != CC_OK) return r;
    const int have = std::min(js[job].sweeps, c->hist_cap);
    if (count) *count = js[job].sweeps;
    const int m = std::min(max, have);
    if (m > 0 && out) {
        CC_CUDA(c, cudaMemcpyAsync(out, c->hist + (size_t)job * c->hist_cap, sizeof(cc_sweep_info) * (size_t)m,
                                   cudaMemcpyDeviceToHost, c->stream));
        CC_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return CC_OK;
}

cc_status cc_sweep(cc_ctx* c, cc_sweep_info* info)
{
    if (!c) return fail(nullptr, CC_ERR_INVALID, "ctx is NULL");
    cc_status r = run(c, 1, nullptr);
    if (r != CC_OK) return r;
    if (info) {
        r = need_single(c);
        if (r != CC_OK) return r;
        std::vector<JobState> js;
        r = read_jobs(c, js);
        if (r != CC_OK) return r;
        const int s = js[0].sweeps;
        if (s >= 1 && s <= c->hist_cap) {
            CC_CUDA(c, cudaMemcpyAsync(info, c->hist + (s - 1), sizeof(cc_sweep_info), cudaMemcpyDeviceToHost, c->stream));
            CC_CUDA(c, cudaStreamSynchronize(c->stream));
        } else {
            std::memset(info, 0, sizeof(*info));
            info->F = js[0].F;
        }
    }
    return CC_OK;
}

cc_status cc_run_until_converged(cc_ctx* c, int32_t max_sweeps, int32_t* sweeps_done)
{
    if (!c) return fail(nullptr, CC_ERR_INVALID, "ctx is NULL");
    int limit = max_sweeps > 0 ? max_sweeps : c->opt.max_sweeps;
    int done = 0;
    cc_status r = run(c, limit, &done);
    if (sweeps_done) *sweeps_done = done;
    return r;
}

cc_status cc_last_run_timing(cc_ctx* c, int32_t max, float* sweep_ms, float* propose_ms, int32_t* count)
{
    if (!c) return fail(nullptr, CC_ERR_INVALID, "ctx is NULL");
    const int have = (int)c->sweep_ms.size();
    if (count) *count = have;
    for (int i = 0; i < have && i < max; ++i) {
        if (sweep_ms) sweep_ms[i] = c->sweep_ms[i];
        if (propose_ms) propose_ms[i] = c->propose_ms[i];
    }
    return CC_OK;
}

cc_status cc_table_stats(cc_ctx* c, cc_table_info* out)
{
    if (!c || !out) return fail(c, CC_ERR_INVALID, "null argument");
    DevState s;
    cc_status r = read_state(c, &s);
    if (r != CC_OK) return r;
    out->capacity = (int64_t)(s.mask + 1);
    out->max_capacity = (int64_t)c->cap_max;
    out->live_keys = s.live;
    out->used_slots = (int64_t)s.used;
    out->rebuilds = s.rebuilds;
    out->retries = s.retries;
    return CC_OK;
}

cc_status cc_launch_count(const cc_ctx* c, int64_t* out)
{
    if (!c || !out) return fail(nullptr, CC_ERR_INVALID, "null argument");
    // kernels outside the sweep graphs' regions are counted here, those of
    // the regions that ran by their gates on the device
    cc_ctx* m = const_cast<cc_ctx*>(c);
    DevState s;
    cc_status r = read_state(m, &s);
    if (r != CC_OK) return r;
    *out = c->launches + (int64_t)s.region_launches;
    return CC_OK;
}

cc_status cc_history(cc_ctx* c, int32_t max, cc_sweep_info* out, int32_t* count)
{
    if (!c) return fail(nullptr, CC_ERR_INVALID, "ctx is NULL");
    cc_status r = need_single(c);
    if (r != CC_OK) return r;
    return cc_job_history(c, 0, max, out, count);
}

cc_status cc_job_objective(cc_ctx* c, int32_t job, int64_t* out, int32_t* sweeps)
{
    cc_status r = check_job(c, job);
    if (r != CC_OK) return r;
    std::vector<JobState> js;
    r = read_jobs(c, js);
    if (r != CC_OK) return r;
    if (out) *out = js[job].F;
    if (sweeps) *sweeps = js[job].sweeps;
    return CC_OK;
}

cc_status cc_objective(cc_ctx* c, int64_t* out)
{
    if (!c || !out) return fail(c, CC_ERR_INVALID, "null argument");
    cc_status r = need_single(c);
    if (r != CC_OK) return r;
    return cc_job_objective(c, 0, out, nullptr);
}

cc_status cc_objective_recompute(cc_ctx* c, int64_t* out)
{
    if (!c || !out) return fail(c, CC_ERR_INVALID, "null argument");
    cc_status r = need_single(c);
    if (r != CC_OK) return r;
    std::vector<long long> F;
    r = objective_recompute(c, F);
    if (r == CC_OK) *out = F[0];
    return r;
}

cc_status cc_cluster_ids(cc_ctx* c, int32_t* out)
{
    if (!c || !out) return fail(c, CC_ERR_INVALID, "null argument");
    const int* src = c->C;
    if (c->jobs > 1) {
        k_shift_ids<<<c->sms * 8, 256, 0, c->stream>>>(c->n, c->C, c->jid, c->d_job, -1, c->scratch);
        c->launches += 1;
        src = c->scratch;
    }
    CC_CUDA(c, cudaMemcpyAsync(out, src, sizeof(int) * (size_t)c->n, cudaMemcpyDeviceToHost, c->stream));
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    return CC_OK;
}

cc_status cc_cluster_ids_dev(cc_ctx* c, const int32_t** out)
{
    if (!c || !out) return fail(c, CC_ERR_INVALID, "null argument");
    *out = c->C;
    return CC_OK;
}

cc_status cc_consensus_labels(cc_ctx* c, int32_t* out)
{
    if (!c || !out) return fail(c, CC_ERR_INVALID, "null argument");
    int* lab = nullptr;
    cc_status r = renumber(c, &lab);
    if (r != CC_OK) return r;
    CC_CUDA(c, cudaMemcpyAsync(out, lab, sizeof(int) * (size_t)c->n, cudaMemcpyDeviceToHost, c->stream));
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    return CC_OK;
}

cc_status cc_job_labels(cc_ctx* c, int32_t job, int32_t* out)
{
    cc_status r = check_job(c, job);
    if (r != CC_OK) return r;
    if (!out) return fail(c, CC_ERR_INVALID, "null argument");
    int* lab = nullptr;
    r = renumber(c, &lab);
    if (r != CC_OK) return r;
    const JobInfo& J = c->job[job];
    CC_CUDA(c, cudaMemcpyAsync(out, lab + J.vo, sizeof(int) * (size_t)J.n, cudaMemcpyDeviceToHost, c->stream));
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    return CC_OK;
}

cc_status cc_batch_run(cc_ctx* c, int32_t max_sweeps)
{
    return cc_run_until_converged(c, max_sweeps, nullptr);
}

cc_status cc_batch_result(cc_ctx* c, int32_t job, int32_t* labels_out, int64_t* objective_out)
{
    if (!c) return fail(nullptr, CC_ERR_INVALID, "ctx is NULL");
    if (!labels_out && !objective_out) return fail(c, CC_ERR_INVALID, "both outputs are NULL");
    cc_status r = CC_OK;
    if (labels_out) r = cc_job_labels(c, job, labels_out);
    if (r == CC_OK && objective_out) r = cc_job_objective(c, job, objective_out, nullptr);
    return r;
}

cc_status cc_metrics(cc_ctx* c, cc_partition_metrics* out)
{
    if (!c || !out) return fail(c, CC_ERR_INVALID, "null argument");
    // a rebuild at the current capacity makes the summary rows exact maxima
    DevState pre;
    cc_status r = read_state(c, &pre);
    if (r != CC_OK) return r;
    if (pre.err) return check_device_error(c, pre);
    CC_CUDA(c, cudaMemcpyAsync(&c->st->new_mask, &pre.mask, sizeof(pre.mask), cudaMemcpyHostToDevice, c->stream));
    CC_CUDA(c, launch_table_rebuild(c->args, c->rows, false, c->stream));
    c->launches += kKernelsPerRebuild;
    const int P = c->parts, J = c->jobs;
    const size_t bytes = sizeof(int) * (size_t)c->nlabels + (sizeof(long long) * 3 + sizeof(double)) * (size_t)P +
                         (sizeof(long long) + sizeof(double)) * (size_t)J + 64;
    unsigned char* buf = nullptr;
    CC_CUDA(c, c->pool ? cudaMallocFromPoolAsync((void**)&buf, bytes, c->pool, c->stream) : cudaMalloc((void**)&buf, bytes));
    MetricsArgs m{};
    long long* sq = reinterpret_cast<long long*>(buf);
    long long* sjc = sq + P;
    long long* sjl = sjc + P;
    long long* csq = sjl + P;
    double* slog = reinterpret_cast<double*>(csq + J);
    double* cslog = slog + P;
    int* lmax = reinterpret_cast<int*>(cslog + J);
    m.pfirst = c->d_pfirst;
    m.lbase = c->d_lbase;
    m.nlabels = c->nlabels;
    m.lmax = lmax;
    m.sq = sq;
    m.slog = slog;
    m.sjc = sjc;
    m.sjl = sjl;
    m.csq = csq;
    m.cslog = cslog;
    std::vector<long long> h_sq(P), h_sjc(P), h_sjl(P), h_csq(J), h_psq(P);
    std::vector<double> h_slog(P), h_cslog(J), h_pslog(P);
    cudaError_t e = cudaMemsetAsync(buf, 0, bytes, c->stream);
    if (e == cudaSuccess) e = launch_metrics(c->args, m, P, c->stream);
    c->launches += 3;
    auto get = [&](void* dst, const void* src, size_t n) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, c->stream);
    };
    get(h_sq.data(), sq, sizeof(long long) * P);
    get(h_sjc.data(), sjc, sizeof(long long) * P);
    get(h_sjl.data(), sjl, sizeof(long long) * P);
    get(h_csq.data(), csq, sizeof(long long) * J);
    get(h_slog.data(), slog, sizeof(double) * P);
    get(h_cslog.data(), cslog, sizeof(double) * J);
    get(h_psq.data(), c->part_sq, sizeof(long long) * P);
    get(h_pslog.data(), c->part_slog, sizeof(double) * P);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (c->pool) cudaFreeAsync(buf, c->stream);
    else cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(c, e, "metrics");
    for (int j = 0; j < J; ++j) {
        const JobInfo& Jb = c->job[j];
        const double n = (double)Jb.n;
        for (int i = 0; i < Jb.k; ++i) {
            const int p = c->pfirst[j] + i;
            cc_partition_metrics& o = out[p];
            o.mirkin = h_csq[j] + h_psq[p] - 2 * h_sq[p];
            o.split_join = 2 * Jb.n - h_sjc[p] - h_sjl[p];
            o.rand_distance = Jb.n > 1 ? (double)o.mirkin / (n * (n - 1.0)) : 0.0;
            o.vi = (h_cslog[j] + h_pslog[p] - 2.0 * h_slog[p]) / n;
        }
    }
    DevState s;
    r = read_state(c, &s);
    if (r != CC_OK) return r;
    return check_device_error(c, s);
}

cc_status cc_partition_distances(cc_ctx* c, cc_partition_metrics* out)
{
    if (!c || !out) return fail(c, CC_ERR_INVALID, "null argument");
    cc_status r = need_single(c);
    if (r != CC_OK) return r;
    const int k = c->job[0].k;
    const long long n = c->n;
    DevState pre;
    r = read_state(c, &pre);
    if (r != CC_OK) return r;
    if (pre.err) return check_device_error(c, pre);
    // the consensus is kept aside and restored; each input partition in turn
    // becomes the consensus, and the distance reductions give its row
    int* saved = c->scratch;
    CC_CUDA(c, cudaMemcpyAsync(saved, c->C, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, c->stream));
    const unsigned long long full = c->cap_max - 1;
    std::vector<cc_partition_metrics> row(k);
    for (int a = 0; a < k && r == CC_OK; ++a) {
        CC_CUDA(c, launch_ids_from_partition(c->args, n, 0, a, c->stream));
        CC_CUDA(c, launch_state_from_ids(c->args, c->stream));
        CC_CUDA(c, cudaMemcpyAsync(&c->st->mask, &full, sizeof(full), cudaMemcpyHostToDevice, c->stream));
        c->launches += 3;
        r = cc_metrics(c, row.data());
        for (int i = 0; r == CC_OK && i < k; ++i) out[(size_t)a * k + i] = row[i];
    }
    // restore C, its sizes and its table at the capacity it had
    CC_CUDA(c, cudaMemcpyAsync(c->C, saved, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, c->stream));
    CC_CUDA(c, launch_state_from_ids(c->args, c->stream));
    CC_CUDA(c, cudaMemcpyAsync(&c->st->new_mask, &pre.mask, sizeof(pre.mask), cudaMemcpyHostToDevice, c->stream));
    CC_CUDA(c, launch_table_rebuild(c->args, c->rows, false, c->stream));
    c->launches += 2 + kKernelsPerRebuild;
    if (r != CC_OK) return r;
    DevState s;
    r = read_state(c, &s);
    if (r != CC_OK) return r;
    return check_device_error(c, s);
}

cc_status cc_group_partitions(int32_t k, const int64_t* distance, int64_t lambda, int32_t* group_of,
                              int32_t* groups)
{
    if (k < 1 || !distance || !group_of) return fail(nullptr, CC_ERR_INVALID, "cc_group_partitions needs k >= 1 and arrays");
    std::vector<int> parent(k);
    for (int i = 0; i < k; ++i) parent[i] = i;
    auto root = [&](int x) {
        while (parent[x] != x) x = parent[x] = parent[parent[x]];
        return x;
    };
    for (int a = 0; a < k; ++a)
        for (int b = a + 1; b < k; ++b) {
            // an edge survives unless its weight is above lambda; either triangle counts
            if (distance[(size_t)a * k + b] <= lambda || distance[(size_t)b * k + a] <= lambda) {
                const int ra = root(a), rb = root(b);
                if (ra != rb) parent[ra > rb ? ra : rb] = ra < rb ? ra : rb;
            }
        }
    std::vector<int> id(k, -1);
    int ng = 0;
    for (int i = 0; i < k; ++i) {
        const int ri = root(i);
        if (id[ri] < 0) id[ri] = ng++;
        group_of[i] = id[ri];
    }
    if (groups) *groups = ng;
    return CC_OK;
}

cc_status cc_job_count(const cc_ctx* c, int32_t* out)
{
    if (!c || !out) return fail(nullptr, CC_ERR_INVALID, "null argument");
    *out = c->jobs;
    return CC_OK;
}

const char* cc_last_error(const cc_ctx* c)
{
    return c ? c->err.c_str() : g_create_error.c_str();
}

void cc_destroy(cc_ctx* c)
{
    ctx_destroy(c);
}

}  // extern "C"

namespace ccg {

void set_thread_error(const std::string& msg)
{
    g_create_error = msg;
}

}  // namespace ccg
