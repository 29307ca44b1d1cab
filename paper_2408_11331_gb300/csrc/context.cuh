// Host-side state of a context (cc_ctx) and the internal calls that the
// served form (server.cu) builds on: sizing a set of jobs before creating it,
// creating a context from a memory pool, and running it without blocking.
#pragma once

#include <map>
#include <string>
#include <vector>

#include "cc_internal.cuh"

// A run of `limit` sweeps unrolled into one graph, with events at every sweep
// boundary and around every proposal step.
struct RunGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaEvent_t> bound;    // limit + 1
    std::vector<cudaEvent_t> prop;     // 2 * limit
};

struct cc_ctx {
    int jobs = 0, kmax = 0;
    long long n = 0, nnz = 0, rows = 0, keys = 0;
    int device = 0, sms = 0;
    cudaStream_t stream = nullptr;      // stream used by calls
    cudaStream_t own_stream = nullptr;  // stream created by the context (also used for capture)
    cudaStream_t body_stream = nullptr; // captures the bodies of a sweep graph's conditional regions
    cudaStream_t loop_stream = nullptr; // captures the body of a run loop (batches: a run is one launch)
    bool loop_ok = true;                // the run loop graph could be built (else: chunks of sweeps)
    cudaMemPool_t pool = nullptr;       // device memory comes from this pool (stream-ordered) if set
    std::vector<ccg::JobInfo> job;      // host copy of the job table
    std::vector<long long> F0;          // objective of each job at the singleton start
    std::vector<long long> psq;         // sum_ij |P_ij|^2 of each job
    std::vector<int> pfirst;            // first global partition of each job
    std::vector<long long> eo;          // first CSR entry of each job (jobs + 1)
    // capacity of each job's place in the union (its sizes at creation): a
    // served context can load a smaller job into a place whose job is done
    std::vector<long long> slot_n, slot_nnz;
    std::vector<int> slot_k;
    std::vector<long long> lbase;       // first label id of each job in a job-concatenated id space
    long long nlabels = 0;              // sum_j k_j 2^s_j
    int parts = 0;                      // sum_j k_j
    int* d_pfirst = nullptr;
    long long* d_lbase = nullptr;
    long long* part_sq = nullptr;       // per global partition: sum_l |P_il|^2
    double* part_slog = nullptr;        // per global partition: sum_l |P_il| log |P_il|
    ccg::JobInfo* d_job = nullptr;
    ccg::JobState* js = nullptr;
    long long* off = nullptr;
    int* col = nullptr;
    int* src = nullptr;
    int* jid = nullptr;
    int* G = nullptr;
    int4* summ = nullptr;
    int* C = nullptr;
    int* size = nullptr;
    int* dsize = nullptr;
    unsigned long long* best = nullptr;
    int* aown = nullptr;
    int* chg = nullptr;                 // active set: change stamp per cluster id (n)
    unsigned long long* prev = nullptr; // active set: previous bid per vertex (n)
    unsigned char* act = nullptr;       // active set: scored in this sweep (n)
    ccg::Slot* table = nullptr;
    int* pv = nullptr;
    int* pa = nullptr;
    int* pb = nullptr;
    int* pg = nullptr;
    unsigned char* pflag = nullptr;
    int* members = nullptr;             // rebuild scratch (n)
    int* cursor = nullptr;              // rebuild scratch (n)
    int* bsum = nullptr;                // rebuild scratch (n/1024 + 2)
    int* scratch = nullptr;             // 3n + n/1024 + 64 ints: output renumbering, warm starts
    // colour_batched: colour of each vertex, vertices and CSR entries by class
    int* colour = nullptr;
    int* vlist = nullptr;
    int* voff = nullptr;
    int* eidx = nullptr;
    long long* eoff = nullptr;
    long long* ccnt = nullptr;          // colouring scratch (2 (n + 2)) and a flag
    int ncls = 1;                       // colour classes (1 without colour_batched)
    bool tuned = true;                  // autotune: lanes chosen (or not to be tuned)
    ccg::DevState* st = nullptr;
    cc_sweep_info* hist = nullptr;
    int hist_cap = 0;
    ccg::SweepArgs args{};
    std::map<int, RunGraph> graphs;     // key > 0: chunk of that many bodies; key < 0: run loop of that limit
    std::vector<float> sweep_ms;        // device time of each sweep of the last run
    std::vector<float> propose_ms;      // ... and of its proposal kernels
    long long launches = 0;             // kernels launched so far
    int grid = 0;
    unsigned long long cap_start = 0;   // active table capacity at the singleton start
    unsigned long long cap_max = 0;     // allocated table capacity
    bool started = false;               // start_state ran once
    cc_options opt{};
    std::vector<void*> allocs;
    size_t bytes = 0;                   // device bytes held
    std::string err;
    // a run driven without blocking (ctx_async_*)
    ccg::DevState* hstate = nullptr;    // pinned host copy of st, owned by the caller
    ccg::JobState* hjobs = nullptr;     // pinned host copy of the job records, owned by the caller (or null)
    cudaEvent_t chunk_done = nullptr;   // recorded after each graph launch and the copy of st
    int async_limit = 0;
    int async_launches = 0;
};

namespace ccg {

// One input job, pointers host or device.
struct JobInput {
    int32_t n;
    int64_t nnz;
    const int64_t* row_off;
    const int32_t* col;
    int32_t k;
    const int32_t* labels;
};

// Sizes of a context for a set of jobs, and the device bytes it holds.
struct Plan {
    int jobs = 0, kmax = 0, hist_cap = 0;
    long long n = 0, nnz = 0, rows = 0, keys = 0, parts = 0;
    unsigned long long cap_max = 0, cap_start = 0, lcap = 0;
    size_t persistent = 0;  // held until cc_destroy
    size_t temporary = 0;   // held during creation only
};

// Checks the sizes of the jobs and the options (host only; the data pointers
// are not looked at) and sizes the context; *msg gets the reason of a failure.
cc_status plan_jobs(int jobs, const JobInput* in, const cc_options& opt, Plan* out, std::string* msg);
cc_status check_options(const cc_options& opt, std::string* msg);
// Fills the capacities and byte counts of a plan from its totals (jobs, n,
// nnz, rows, keys, parts, kmax).
void finish_plan(Plan& p, const cc_options& opt);
// Lanes that score one (vertex, candidate) pair for partitions of count k.
int lanes_for_k(int k);

// Options with the defaults filled in.
cc_options resolve_options(const cc_options* opt);

// cc_create / cc_batch_create with device memory from `pool` (stream-ordered
// allocation on the context's own stream) when pool is not null; the own
// stream gets the given CUDA stream priority (lower numbers run first).
cc_status ctx_create(int jobs, const JobInput* in, bool on_device, const cc_options* opt, void* stream,
                     cudaMemPool_t pool, cc_ctx** out, int priority = 0);

// Starts a run of at most `limit` sweeps without waiting: queues the run and
// its first graph launch, then a copy of the control block into `pinned` and
// an event.
cc_status ctx_async_start(cc_ctx* c, int limit, DevState* pinned, JobState* pinned_jobs = nullptr);

// Checks a run started by ctx_async_start: 0 = still running (the next graph
// launch is queued when the previous one ended without stopping), 1 = every
// job has stopped, -1 = failed (*st holds the status).
int ctx_async_poll(cc_ctx* c, cc_status* st);
// As ctx_async_poll, but when a graph launch ended without stopping the run
// it returns 2 without queueing the next launch: the pinned job records are
// then those after that launch (a job with stop set is done and its labels
// are final), and ctx_async_continue queues the next launch.
int ctx_async_poll_step(cc_ctx* c, cc_status* st);
cc_status ctx_async_continue(cc_ctx* c);

// Whether a job of these sizes fits the place of job j (see ctx_load_job):
// no more vertices, CSR entries, partitions, label rows or keys than the
// place, and at least a quarter of its vertices and CSR entries.
bool ctx_slot_fits(const cc_ctx* c, int j, const JobInput& in);

// Loads a new job into the place of job j, whose run has ended and whose
// results were taken, while the context's other jobs keep running: the CSR,
// the compacted labels and the singleton state of the new job go into job
// j's ranges (vertices the new job does not use go to an idle job that
// never runs; CSR entries it does not use become self-loops of its last
// vertex, which the method ignores), job j's record restarts at the new
// job's singleton start, the finished job's contingency keys get count 0
// and the new job's singleton keys are inserted (only if the table runs
// short is it rebuilt from C, in the next sweep).  The new job's results are
// then those of running it alone.  Host inputs are read before the call returns.  The run goes on
// with ctx_async_continue.  Errors: CC_ERR_INVALID (malformed input; the
// context is unchanged), CC_ERR_OOM, CC_ERR_CUDA.
cc_status ctx_load_job(cc_ctx* c, int j, const JobInput& in);

// Labels of job j alone, renumbered as by cc_job_labels, into host memory
// (blocks until they are there).  Valid once the job has stopped, also
// while other jobs of the context still run.
cc_status ctx_job_labels_now(cc_ctx* c, int j, int32_t* out);

// Objective and sweeps of every job (synchronises the context's stream).
cc_status ctx_job_results(cc_ctx* c, std::vector<long long>& F, std::vector<int>& sweeps);

// Renumbered labels of job j into host memory (queued on the context's
// stream; synchronise before reading).
cc_status ctx_copy_labels(cc_ctx* c, const int* dev_labels, int j, int32_t* out);

// Renumbers the labels of every job on the device; *dev_labels points into
// the context's scratch.
cc_status ctx_renumber(cc_ctx* c, int** dev_labels);

void ctx_destroy(cc_ctx* c);

}  // namespace ccg
