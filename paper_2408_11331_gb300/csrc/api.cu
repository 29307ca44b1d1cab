// The C ABI declared in include/cc.h: context lifetime, the sweep loop as a
// captured CUDA graph, and the output calls.
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "cc_internal.cuh"

using namespace ccg;

// A run of `limit` sweeps unrolled into one graph, with events at every sweep
// boundary and around every proposal launch.
struct RunGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaEvent_t> bound;    // limit + 1
    std::vector<cudaEvent_t> prop;     // 2 * limit
};

struct cc_ctx {
    int n = 0, k = 0, kp = 0, lshift = 0;
    long long nnz = 0;
    int device = 0, sms = 0;
    cudaStream_t stream = nullptr;      // stream used by calls
    cudaStream_t own_stream = nullptr;  // stream created by the context (also used for capture)
    long long* off = nullptr;
    int* col = nullptr;
    int* src = nullptr;                 // source vertex of each CSR entry
    int* G = nullptr;
    int* C = nullptr;
    int* size = nullptr;
    int* dsize = nullptr;
    unsigned long long* best = nullptr;
    int* aown = nullptr;                // A_a per vertex (proposal step)
    Slot* table = nullptr;
    int* pv = nullptr;
    int* pa = nullptr;
    int* pb = nullptr;
    int* pg = nullptr;
    unsigned char* pflag = nullptr;
    unsigned int* pslot = nullptr;
    int* scratch = nullptr;             // 3n + n/1024 + 64 ints for the output renumbering
    int* members = nullptr;             // rebuild scratch (n)
    int4* summ = nullptr;               // per-cluster label summaries (n x kp)
    int* cursor = nullptr;              // rebuild scratch (n)
    int* bsum = nullptr;                // rebuild scratch (n/1024 + 2)
    DevState* st = nullptr;
    cc_sweep_info* hist = nullptr;
    int hist_cap = 1 << 16;
    SweepArgs args{};
    std::map<int, RunGraph> graphs;
    std::vector<float> sweep_ms;        // device time of each sweep of the last run
    std::vector<float> propose_ms;      // ... and of its proposal kernels
    long long launches = 0;             // kernels launched so far
    int grid = 0;
    long long partition_sq = 0, F0 = 0;
    unsigned long long cap_start = 0;   // active table capacity at the singleton start
    unsigned long long cap_max = 0;     // allocated table capacity
    bool started = false;               // start_state ran once
    cc_options opt{};
    std::vector<void*> allocs;
    std::string err;
};

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
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
    if (e != cudaSuccess) return e;
    c->allocs.push_back(q);
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
    for (void* p : c->allocs) cudaFree(p);
    c->allocs.clear();
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    c->own_stream = nullptr;
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

cc_status check_device_error(cc_ctx* c, const DevState& s)
{
    if (s.err == CC_ERR_TABLE_FULL) return fail(c, CC_ERR_TABLE_FULL, "contingency hash is full");
    if (s.err == CC_ERR_INVALID) return fail(c, CC_ERR_INVALID, "inconsistent contingency state");
    if (s.err != 0) return fail(c, (cc_status)s.err, "device-side failure");
    return CC_OK;
}

cc_status objective_recompute(cc_ctx* c, long long* out)
{
    DevState pre;
    cc_status rp = read_state(c, &pre);
    if (rp != CC_OK) return rp;
    if (!pre.tvalid) {
        // no table yet (singleton start): build it from C first
        CC_CUDA(c, cudaMemcpyAsync(&c->st->new_mask, &pre.mask, sizeof(pre.mask), cudaMemcpyHostToDevice, c->stream));
        CC_CUDA(c, launch_table_rebuild(c->args, false, c->stream));
        c->launches += kKernelsPerRebuild;
    }
    CC_CUDA(c, launch_objective_recompute(c->args, c->stream));
    c->launches += 1;
    DevState s;
    cc_status r = read_state(c, &s);
    if (r != CC_OK) return r;
    *out = s.recompute + c->partition_sq;
    return CC_OK;
}

// Singleton start: C[v] = v, sizes 1, table rebuilt, F = F0, history cleared.
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
    }
    c->started = true;
    s.partition_sq = c->partition_sq;
    s.F = c->F0;
    s.stop = 1;
    s.new_mask = c->cap_start - 1;
    s.mask = c->cap_start - 1;
    CC_CUDA(c, cudaMemcpyAsync(c->st, &s, sizeof(s), cudaMemcpyHostToDevice, c->stream));
    CC_CUDA(c, launch_init_state(c->args, c->stream));
    if (c->opt.sweep_mode == 1) {
        // staged deltas need the singleton counts in the table from the start
        CC_CUDA(c, launch_table_rebuild(c->args, false, c->stream));
        c->launches += 1 + kKernelsPerRebuild;
    } else {
        // the first sweep rebuilds the table itself (it is always heavy);
        // the summary rows of singletons follow from the label rows
        CC_CUDA(c, launch_singleton_summaries(c->args, c->stream));
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
    if (c->graphs.size() >= 8) {  // keep a few limits; drop the others
        for (auto& kv : c->graphs) destroy_graph(kv.second);
        c->graphs.clear();
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
        if (e == cudaSuccess) e = launch_sweep(c->args, c->grid, c->own_stream, g.prop[2 * s], g.prop[2 * s + 1]);
    }
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(g.bound[limit], c->own_stream, cudaEventRecordExternal);
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

// Sweeps per graph launch: a run launches the graph until the device says the
// run has stopped, so at most kChunk - 1 skipped sweep bodies are submitted
// after the last sweep (each costs its kernels' launch latency).
constexpr int kChunk = 4;

cc_status run(cc_ctx* c, int limit, int* done)
{
    const int chunk = limit < kChunk ? limit : kChunk;
    RunGraph* g = nullptr;
    cc_status r = ensure_graph(c, chunk, &g);
    if (r != CC_OK) return r;
    CC_CUDA(c, launch_run_begin(c->st, limit, c->stream));
    c->launches += 1;
    c->sweep_ms.clear();
    c->propose_ms.clear();
    DevState st;
    int before = 0;
    // a sweep abandoned for lack of table space is retried in the next body,
    // so the number of launches is bounded by the limit plus the retries
    for (int launch = 0; launch < limit + 64; ++launch) {
        CC_CUDA(c, cudaGraphLaunch(g->exec, c->stream));
        c->launches += (long long)chunk * kKernelsPerSweep;
        r = read_state(c, &st);
        if (r != CC_OK) return r;
        const int ran = st.run_sweeps - before;
        for (int b = 0; b < ran && b < chunk; ++b) {
            float x = 0.f, y = 0.f;
            CC_CUDA(c, cudaEventElapsedTime(&x, g->bound[b], g->bound[b + 1]));
            CC_CUDA(c, cudaEventElapsedTime(&y, g->prop[2 * b], g->prop[2 * b + 1]));
            c->sweep_ms.push_back(x);
            c->propose_ms.push_back(y);
        }
        before = st.run_sweeps;
        if (st.stop || st.err) break;
    }
    r = check_device_error(c, st);
    if (r != CC_OK) return r;
    if (!st.stop) return fail(c, CC_ERR_TABLE_FULL, "sweep retries did not converge");
    if (done) *done = st.run_sweeps;
    if (c->opt.debug_checks) {
        long long F = 0;
        r = objective_recompute(c, &F);
        if (r != CC_OK) return r;
        if (F != st.F) return fail(c, CC_ERR_INVALID, "debug check: incremental objective differs from recomputed");
    }
    return CC_OK;
}

cc_status create_common(int32_t n, int64_t nnz, const int64_t* row_off, const int32_t* col, int32_t k,
                        const int32_t* labels, bool on_device, const cc_options* opt, void* stream,
                        cc_ctx** out)
{
    if (!out) return fail(nullptr, CC_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (n < 1) return fail(nullptr, CC_ERR_INVALID, "n must be >= 1");
    if (k < 1) return fail(nullptr, CC_ERR_INVALID, "k must be >= 1");
    if (k > 4096) return fail(nullptr, CC_ERR_INVALID, "k must be <= 4096");
    if (nnz < 0) return fail(nullptr, CC_ERR_INVALID, "nnz must be >= 0");
    if (!row_off || !labels || (nnz > 0 && !col)) return fail(nullptr, CC_ERR_INVALID, "null input pointer");
    if (3LL * k * n + k >= (1LL << 31)) return fail(nullptr, CC_ERR_OVERFLOW, "3 k n + k >= 2^31");
    if (opt) {
        for (int r : opt->reserved)
            if (r != 0) return fail(nullptr, CC_ERR_INVALID, "reserved option fields must be zero");
        if (opt->table_log2 < 0 || opt->table_log2 > 40) return fail(nullptr, CC_ERR_INVALID, "table_log2 out of range");
        if (opt->table_start_log2 < 0 || opt->table_start_log2 > 40)
            return fail(nullptr, CC_ERR_INVALID, "table_start_log2 out of range");
        if (opt->sweep_mode < 0 || opt->sweep_mode > 2) return fail(nullptr, CC_ERR_INVALID, "sweep_mode must be 0, 1 or 2");
    }

    cc_ctx* c = new cc_ctx();
    c->n = n;
    c->k = k;
    c->kp = (k + 3) & ~3;
    while ((1LL << c->lshift) < n) ++c->lshift;
    c->nnz = nnz;
    if (opt) c->opt = *opt;
    else cc_default_options(&c->opt);
    if (c->opt.max_sweeps <= 0) c->opt.max_sweeps = 20;

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
    CC_TRY(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking));
    c->stream = stream ? static_cast<cudaStream_t>(stream) : c->own_stream;

    const unsigned long long kn = (unsigned long long)k * n;
    unsigned long long cap = c->opt.table_log2 > 0 ? (1ull << c->opt.table_log2) : next_pow2(4 * kn + 64);
    if (cap < 64) cap = 64;

    CC_TRY(dalloc(c, &c->off, (size_t)n + 1));
    CC_TRY(dalloc(c, &c->col, (size_t)nnz));
    CC_TRY(dalloc(c, &c->src, (size_t)nnz));
    CC_TRY(dalloc(c, &c->aown, (size_t)n));
    CC_TRY(dalloc(c, &c->G, (size_t)n * c->kp));
    CC_TRY(dalloc(c, &c->C, (size_t)n));
    CC_TRY(dalloc(c, &c->size, (size_t)n));
    CC_TRY(dalloc(c, &c->dsize, (size_t)n));
    CC_TRY(dalloc(c, &c->best, (size_t)n));
    CC_TRY(dalloc(c, &c->table, (size_t)cap));
    CC_TRY(dalloc(c, &c->pv, (size_t)n));
    CC_TRY(dalloc(c, &c->pa, (size_t)n));
    CC_TRY(dalloc(c, &c->pb, (size_t)n));
    CC_TRY(dalloc(c, &c->pg, (size_t)n));
    CC_TRY(dalloc(c, &c->pflag, (size_t)n));
    CC_TRY(dalloc(c, &c->pslot, 2 * (size_t)kn));
    CC_TRY(dalloc(c, &c->scratch, 3 * (size_t)n + (size_t)n / 1024 + 64));
    CC_TRY(dalloc(c, &c->members, (size_t)n));
    CC_TRY(dalloc(c, &c->summ, (size_t)n * c->kp));
    CC_TRY(dalloc(c, &c->cursor, (size_t)n));
    CC_TRY(dalloc(c, &c->bsum, (size_t)n / 1024 + 2));
    CC_TRY(dalloc(c, &c->st, 1));
    CC_TRY(dalloc(c, &c->hist, (size_t)c->hist_cap));

    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CC_TRY(cudaMemcpyAsync(c->off, row_off, sizeof(long long) * ((size_t)n + 1), kind, c->stream));
    if (nnz > 0) CC_TRY(cudaMemcpyAsync(c->col, col, sizeof(int) * (size_t)nnz, kind, c->stream));

    DevState s0;
    std::memset(&s0, 0, sizeof(s0));
    CC_TRY(cudaMemcpyAsync(c->st, &s0, sizeof(s0), cudaMemcpyHostToDevice, c->stream));
    CC_TRY(launch_validate(n, nnz, c->off, c->col, c->st, c->stream));
    DevState s;
    if (read_state(c, &s) != CC_OK) return bail(CC_ERR_CUDA);
    if (s.err) return bail(fail(c, CC_ERR_INVALID, "malformed CSR: offsets must start at 0, end at nnz and not decrease; columns must lie in [0, n)"));
    CC_TRY(launch_fill_src(n, c->off, c->src, c->stream));

    // label compaction (scratch: the label map and, for host input, a device copy)
    {
        int* dlabels = nullptr;
        void* lmap = nullptr;
        const unsigned long long lcap = next_pow2(2 * kn + 64);
        cudaError_t e = cudaSuccess;
        if (!on_device) {
            e = cudaMalloc(&dlabels, sizeof(int) * kn);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dlabels, labels, sizeof(int) * kn, cudaMemcpyHostToDevice, c->stream);
        }
        if (e == cudaSuccess) e = cudaMalloc(&lmap, 16 * lcap);
        if (e == cudaSuccess)
            e = launch_compact_labels(n, k, c->kp, c->lshift, on_device ? labels : dlabels, c->G, lmap, lcap - 1, c->st,
                                      c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (dlabels) cudaFree(dlabels);
        if (lmap) cudaFree(lmap);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "label compaction"));
    }
    if (read_state(c, &s) != CC_OK) return bail(CC_ERR_CUDA);
    if (s.err) return bail(fail(c, CC_ERR_INVALID, "label compaction failed"));
    c->partition_sq = s.partition_sq;
    c->F0 = c->partition_sq - (long long)k * n;
    c->cap_start = c->opt.table_start_log2 > 0 ? (1ull << c->opt.table_start_log2) : next_pow2(2 * kn + 64);
    if (c->cap_start > cap) c->cap_start = cap;
    c->cap_max = cap;

    SweepArgs& a = c->args;
    a.n = n;
    a.k = k;
    a.kp = c->kp;
    a.nnz = nnz;
    a.off = c->off;
    a.col = c->col;
    a.src = c->src;
    a.aown = c->aown;
    a.G = c->G;
    a.C = c->C;
    a.size = c->size;
    a.dsize = c->dsize;
    a.best = c->best;
    a.table = c->table;
    a.summ = c->summ;
    a.lshift = c->lshift;
    a.sweep_mode = c->opt.sweep_mode;
    a.mask_max = cap - 1;
    a.cap_min = cap < 1024 ? cap : 1024;
    a.pv = c->pv;
    a.pa = c->pa;
    a.pb = c->pb;
    a.pg = c->pg;
    a.pflag = c->pflag;
    a.pslot = c->pslot;
    a.members = c->members;
    a.cursor = c->cursor;
    a.bsum = c->bsum;
    a.st = c->st;
    a.hist = c->hist;
    a.hist_cap = c->hist_cap;

    int per_sm = 0;
    CC_TRY(prepare_propose(c->kp, &per_sm));
    if (per_sm < 1) return bail(fail(c, CC_ERR_INVALID, "proposal kernel cannot be resident for this k"));
    c->grid = c->sms * per_sm;

    cc_status rc = start_state(c);
    if (rc != CC_OK) return bail(rc);
    *out = c;
    return CC_OK;
#undef CC_TRY
}

// Output renumbering: first[c] = least vertex of cluster c; flag[first[c]] = 1;
// rank = exclusive prefix sum of flags; label[v] = rank[first[C[v]]].
__global__ void k_first(int n, int* first)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) first[v] = 0x7fffffff;
}

__global__ void k_first_min(int n, const int* __restrict__ C, int* first)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) atomicMin(&first[C[v]], (int)v);
}

// flag[v] = 1 iff v is the least vertex of its cluster; per-block counts.
__global__ void k_flags(int n, const int* __restrict__ C, const int* __restrict__ first, int* flag, int* blocksum)
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
__global__ void k_scan_blocks(int nb, int* blocksum)
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
__global__ void k_rank(int n, int* flag, const int* blocksum)
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

__global__ void k_relabel(int n, const int* __restrict__ C, const int* __restrict__ first,
                          const int* __restrict__ rank, int* out)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) out[v] = rank[first[C[v]]];
}

}  // namespace

extern "C" {

void cc_default_options(cc_options* opt)
{
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->max_sweeps = 20;
}

cc_status cc_create(int32_t n, int64_t nnz, const int64_t* row_off, const int32_t* col, int32_t k,
                    const int32_t* labels, const cc_options* opt, cc_ctx** out)
{
    return create_common(n, nnz, row_off, col, k, labels, false, opt, nullptr, out);
}

cc_status cc_create_dev(int32_t n, int64_t nnz, const int64_t* row_off_dev, const int32_t* col_dev, int32_t k,
                        const int32_t* labels_dev, const cc_options* opt, void* stream, cc_ctx** out)
{
    return create_common(n, nnz, row_off_dev, col_dev, k, labels_dev, true, opt, stream, out);
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
    CC_CUDA(c, cudaMemcpyAsync(c->scratch, C, sizeof(int) * (size_t)c->n, cudaMemcpyHostToDevice, c->stream));
    DevState s;
    cc_status r = read_state(c, &s);
    if (r != CC_OK) return r;
    // ids are checked before the context's own state is touched
    CC_CUDA(c, cudaMemsetAsync(&c->st->err, 0, sizeof(int), c->stream));
    SweepArgs probe = c->args;
    probe.C = c->scratch;
    probe.size = c->scratch + c->n;
    probe.dsize = c->scratch + 2 * (size_t)c->n;
    CC_CUDA(c, launch_state_from_ids(probe, c->stream));
    c->launches += 2;
    DevState chk;
    r = read_state(c, &chk);
    if (r != CC_OK) return r;
    if (chk.err) {
        CC_CUDA(c, cudaMemcpyAsync(&c->st->err, &s.err, sizeof(int), cudaMemcpyHostToDevice, c->stream));
        CC_CUDA(c, cudaStreamSynchronize(c->stream));
        return fail(c, CC_ERR_INVALID, "cluster ids must lie in [0, n)");
    }
    CC_CUDA(c, cudaMemcpyAsync(c->C, c->scratch, sizeof(int) * (size_t)c->n, cudaMemcpyDeviceToDevice, c->stream));
    const unsigned long long nm = c->cap_start - 1;
    CC_CUDA(c, cudaMemcpyAsync(&c->st->new_mask, &nm, sizeof(nm), cudaMemcpyHostToDevice, c->stream));
    CC_CUDA(c, launch_state_from_ids(c->args, c->stream));
    CC_CUDA(c, launch_table_rebuild(c->args, false, c->stream));
    c->launches += 2 + kKernelsPerRebuild;
    long long F = 0;
    r = objective_recompute(c, &F);
    if (r != CC_OK) return r;
    CC_CUDA(c, cudaMemcpyAsync(&c->st->F, &F, sizeof(long long), cudaMemcpyHostToDevice, c->stream));
    int one = 1;
    CC_CUDA(c, cudaMemcpyAsync(&c->st->stop, &one, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    DevState after;
    r = read_state(c, &after);
    if (r != CC_OK) return r;
    return check_device_error(c, after);
}

cc_status cc_sweep(cc_ctx* c, cc_sweep_info* info)
{
    if (!c) return fail(nullptr, CC_ERR_INVALID, "ctx is NULL");
    cc_status r = run(c, 1, nullptr);
    if (r != CC_OK) return r;
    if (info) {
        DevState s;
        r = read_state(c, &s);
        if (r != CC_OK) return r;
        if (s.sweeps >= 1 && s.sweeps <= c->hist_cap) {
            CC_CUDA(c, cudaMemcpyAsync(info, c->hist + (s.sweeps - 1), sizeof(cc_sweep_info), cudaMemcpyDeviceToHost, c->stream));
            CC_CUDA(c, cudaStreamSynchronize(c->stream));
        } else {
            std::memset(info, 0, sizeof(*info));
            info->F = s.F;
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
    *out = c->launches;
    return CC_OK;
}

cc_status cc_history(cc_ctx* c, int32_t max, cc_sweep_info* out, int32_t* count)
{
    if (!c) return fail(nullptr, CC_ERR_INVALID, "ctx is NULL");
    DevState s;
    cc_status r = read_state(c, &s);
    if (r != CC_OK) return r;
    int have = s.sweeps < c->hist_cap ? s.sweeps : c->hist_cap;
    if (count) *count = s.sweeps;
    int m = max < have ? max : have;
    if (m > 0 && out) {
        CC_CUDA(c, cudaMemcpyAsync(out, c->hist, sizeof(cc_sweep_info) * (size_t)m, cudaMemcpyDeviceToHost, c->stream));
        CC_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return CC_OK;
}

cc_status cc_objective(cc_ctx* c, int64_t* out)
{
    if (!c || !out) return fail(c, CC_ERR_INVALID, "null argument");
    DevState s;
    cc_status r = read_state(c, &s);
    if (r != CC_OK) return r;
    *out = s.F;
    return CC_OK;
}

cc_status cc_objective_recompute(cc_ctx* c, int64_t* out)
{
    if (!c || !out) return fail(c, CC_ERR_INVALID, "null argument");
    long long F = 0;
    cc_status r = objective_recompute(c, &F);
    if (r == CC_OK) *out = F;
    return r;
}

cc_status cc_cluster_ids(cc_ctx* c, int32_t* out)
{
    if (!c || !out) return fail(c, CC_ERR_INVALID, "null argument");
    CC_CUDA(c, cudaMemcpyAsync(out, c->C, sizeof(int) * (size_t)c->n, cudaMemcpyDeviceToHost, c->stream));
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
    const int n = c->n;
    int* first = c->scratch;
    int* rank = c->scratch + n;
    int* lab = c->scratch + 2 * (size_t)n;
    int* blocksum = c->scratch + 3 * (size_t)n;
    const int nb = (n + 1023) / 1024;
    const int g = c->sms * 8;
    k_first<<<g, 256, 0, c->stream>>>(n, first);
    k_first_min<<<g, 256, 0, c->stream>>>(n, c->C, first);
    k_flags<<<nb, 1024, 0, c->stream>>>(n, c->C, first, rank, blocksum);
    k_scan_blocks<<<1, 1024, 0, c->stream>>>(nb, blocksum);
    k_rank<<<nb, 1024, 0, c->stream>>>(n, rank, blocksum);
    k_relabel<<<g, 256, 0, c->stream>>>(n, c->C, first, rank, lab);
    c->launches += 6;
    CC_CUDA(c, cudaGetLastError());
    CC_CUDA(c, cudaMemcpyAsync(out, lab, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    return CC_OK;
}

const char* cc_last_error(const cc_ctx* c)
{
    return c ? c->err.c_str() : g_create_error.c_str();
}

void cc_destroy(cc_ctx* c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

}  // extern "C"

namespace ccg {

void set_thread_error(const std::string& msg)
{
    g_create_error = msg;
}

}  // namespace ccg
