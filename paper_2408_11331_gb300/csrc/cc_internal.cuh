// Internal declarations shared by the CUDA translation units of libcc.so.
//
// A context holds J independent consensus jobs as one disjoint union (a
// single job is J = 1).  Vertices of job j are the union ids vo_j .. vo_j+n_j-1;
// cluster ids are union vertex ids (the founding vertex), so they never clash
// across jobs and a cluster id also names its job.  Every step of a sweep runs
// over the whole union in the same kernels; each job keeps its own counters,
// guard decisions, objective, convergence and history, so a job's run is
// identical to running it alone.
//
// Device data layout:
//   off   int64[N+1]   union CSR row offsets      col  int32[NNZ] union neighbour ids
//   src   int32[NNZ]   source vertex of each CSR entry
//   jid   int32[N]     job of each vertex (and of each cluster id)
//   G     int32[...]   compacted label ids, vertex-major: job j's rows start at go_j,
//                      kp_j = k_j rounded up to 4 ints each (16-byte rows, padding -1);
//                      g = (i << s_j) | rep, rep the job-local index of the least vertex
//                      carrying that label in partition i and 2^s_j >= n_j, so g names
//                      (partition, label) within the job and g < 2 k_j n_j.
//   summ  int4[...]    same layout as G, one row per cluster id: per partition i
//                      {d1, m1, d2, m2}: the two label ids that were most frequent in the
//                      cluster at the last table rebuild (d1 first; -1 where the cluster
//                      had fewer labels) and the exact current counts of each (kept by
//                      every commit), so |cluster| - m1 - m2 bounds the count of any
//                      other label (and is 0 when d1 and d2 cover the cluster).  The
//                      first 8 bytes read as one unsigned 64-bit value are m1 << 32 | d1
//                      (likewise the last 8), the order in which the rebuild ranks labels.
//   C     int32[N]     cluster id of each vertex
//   size  int32[N]     cluster sizes, indexed by cluster id
//   table Slot[cap]    the contingency counts n(c, i, l) of all jobs as one open-
//                      addressing hash with linear probing, key = c << 32 | g.  Only an
//                      active prefix of st->mask + 1 slots is used; it is rebuilt from C
//                      (with dead keys dropped) when needed.
#pragma once

#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "cc.h"

namespace ccg {

constexpr unsigned long long kEmpty = ~0ull;
constexpr int kWarpsPerBlock = 8;
constexpr int kBlock = kWarpsPerBlock * 32;

// One contingency entry: the (cluster, label id) key, its count and the
// delta staged by the current sweep.  16 bytes, read as one vector load.
struct __align__(16) Slot {
    unsigned long long key;
    int cnt;
    int dlt;
};

// Static description of a job inside the union.
struct JobInfo {
    long long vo;   // first union vertex
    long long n;    // vertices
    long long go;   // first entry of the job's rows in G and summ
    int k;          // input partitions
    int kp;         // k rounded up to 4
    int lshift;     // s_j
    int pad;
};

// Per-job state of the current run.
struct JobState {
    unsigned long long nprop;  // |P| of the current sweep
    unsigned long long np1;    // |P1|
    unsigned long long moves;  // moves committed in the current sweep
    long long dF;              // objective change of the current sweep
    long long dF_p1;           // dF of P1 as evaluated
    long long F;               // current objective
    long long recompute;       // F' accumulator (heavy sweeps, recompute)
    long long partition_sq;    // sum_i sum_j |P_ij|^2
    long long t_prop;          // colour_batched: the sweep's totals over its classes so far:
    long long t_p1;            //   |P|, |P1|, dF of P1, classes that fell back, moves
    long long t_dFp1;
    long long t_fb;
    long long t_moves;
    int mode;                  // 0 nothing to commit, 1 commit P1 (staged), 2 matching, 3 P1 committed (rebuilt)
    int stop;                  // 1: this job's run has stopped
    int sweeps;                // sweeps recorded since creation / reset
    int run_sweeps;            // sweeps in the current run
    int rollback;              // 1: this heavy sweep's P1 was rejected and is being undone
    int pad;
};

// Device-resident control block of a context (union-wide state).
struct DevState {
    unsigned long long nprop;    // proposals of the current sweep, all jobs
    unsigned long long pkeys;    // sum over those proposals of their job's k (label rows they move)
    unsigned long long used;     // occupied table slots
    long long live;              // keys with a non-zero count
    unsigned long long mask;     // active table capacity - 1 (a power of two minus one)
    unsigned long long new_mask; // capacity - 1 of a pending rebuild
    int skip;                    // 1: this sweep does nothing (every job has stopped)
    int stop;                    // 1: the run has stopped (all jobs)
    int active;                  // jobs still running after the current sweep
    int rebuild;                 // 1: a table rebuild is pending
    int err;                     // cc_status of a device-side failure (first one wins)
    int overflow;                // 1: the table ran short during this sweep (nothing committed)
    int abort;                   // 1: the pending rebuild follows an abandoned sweep
    int retries;                 // sweeps abandoned and retried in a larger table
    int rebuilds;                // table rebuilds since creation
    int heavy;                   // 1: this sweep evaluates P1 by a rebuild (see sweep.cu)
    int rollback;                // 1: some job's heavy P1 is being undone
    int tvalid;                  // 1: the table holds the counts of the current C
    int run_limit;               // sweep limit of the current run
    int run_bodies;              // sweeps of the current run that did work (retried ones included)
    unsigned long long region_launches;  // kernels run inside the gated regions of sweep graphs
    int stamp;                   // number of the current sweep (since creation; retried sweeps reuse it)
    int all_active;              // 1: every vertex is scored in this sweep (first sweep of a run)
    int cls;                     // colour_batched: the class this sweep body runs
    int ncls;                    // colour_batched: number of classes (of the job with the most)
    unsigned long long safe_mask;  // heavy sweep: capacity - 1 that holds every key it can create
    int tight;                   // 1: the pending rebuild tries a capacity below safe_mask (checked)
    int again;                   // 1: the tight attempt was too small; the rebuild runs again at safe_mask
    int build_fail;              // 1: an insert of the tight attempt ran past its probe limit
};

// Arguments of the kernels (passed by value).
struct SweepArgs {
    long long n;                // N, union vertices
    long long nnz;              // union CSR entries
    int jobs;                   // J
    int kmax;                   // largest k_j
    const long long* off;
    const int* col;
    const int* src;             // source vertex of each CSR entry (nnz)
    const int* jid;             // job of each vertex
    const JobInfo* job;         // J
    JobState* js;               // J
    const int* G;
    int4* summ;
    int* C;
    int* size;
    int* dsize;                 // staged size deltas
    unsigned long long* best;   // bids: per vertex in the proposal step, per cluster in the matching
    int* aown;                  // A_a of each vertex for the current sweep
    Slot* table;
    unsigned long long mask_max; // allocated capacity - 1; the active capacity is st->mask + 1
    unsigned long long cap_min;  // smallest active capacity
    unsigned long long keys;     // sum_j k_j n_j: no C has more live keys
    int sweep_mode;              // 0 automatic, 1 always staged deltas, 2 always rebuild
    int gs;                      // lanes that score one item (a power of two, 1..32)
    int active_set;              // 1: score only the active vertices (cc_options.active_set)
    int empty_moves;             // 1: a vertex may also move into a new cluster with its own id (cc_options.empty_moves)
    int tight_mode;              // cc_options.tight_rebuild: 0 tight attempt first, 1 never, 2 always dropped
    int colour_mode;             // 1: colour-batched sweeps (cc_options.colour_batched): a sweep body
                                 //    runs the vertices of colour class st->cls only
    const int* vlist;            // colour_batched: vertices listed class by class (n)
    const int* voff;             // colour_batched: first entry of each class in vlist (ncls + 1)
    const int* eidx;             // colour_batched: CSR entries of each class's vertices, class by class (nnz)
    const long long* eoff;       // colour_batched: first entry of each class in eidx (ncls + 1)
    int* chg;                   // per cluster id: stamp of the last sweep that moved a vertex into or out of it
    unsigned long long* prev;   // per vertex: its bid of the last sweep that scored it (kEmpty: none)
    unsigned char* act;         // per vertex: 1 if all its candidates are scored in this sweep
    int* pv;                    // proposal list: vertex,
    int* pa;                    //   source cluster,
    int* pb;                    //   target cluster,
    int* pg;                    //   gain dD
    unsigned char* pflag;       //   1 if kept by the singleton guard (2: matching winner)
    int* members;               // rebuild scratch: vertices listed cluster by cluster (n)
    int* cursor;                // rebuild scratch: next free position of each cluster (n)
    int* bsum;                  // rebuild scratch: per-block sums of the size scan (n / 1024 + 1)
    DevState* st;
    cc_sweep_info* hist;        // J x hist_cap records
    int hist_cap;
};

// Row of vertex / cluster x (a union vertex id) of job J in G or summ.
__device__ __forceinline__ long long row_of(const JobInfo& J, long long x)
{
    return J.go + (x - J.vo) * J.kp;
}

// 64-bit finaliser of MurmurHash3 (Austin Appleby, public domain); used by the
// setup-time label map.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z ^= z >> 33;
    z *= 0xff51afd7ed558ccdull;
    z ^= z >> 33;
    z *= 0xc4ceb9fe1a85ec53ull;
    z ^= z >> 33;
    return z;
}

// Slot hash of a (cluster, label id) key: the two 32-bit halves mixed with odd
// multipliers, then the 32-bit MurmurHash3 finaliser.  Capacities stay below
// 2^32 slots.
__device__ __forceinline__ unsigned long long hash_key(unsigned long long key)
{
    unsigned h = ((unsigned)(key >> 32) * 0x9E3779B1u) ^ ((unsigned)key * 0x85EBCA77u);
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ unsigned long long ckey(int c, int g)
{
    return ((unsigned long long)(unsigned)c << 32) | (unsigned)g;
}

// Keeps the summary row of the slot's (cluster, partition) exact after its
// count changed by d: only the counts of the row's two labels are stored.
__device__ __forceinline__ void summ_update(const SweepArgs& a, unsigned long long key, int d)
{
    const int x = (int)(key >> 32), g = (int)(unsigned)(key & 0xffffffffull);
    const JobInfo& J = a.job[a.jid[x]];
    int4* S = a.summ + row_of(J, x) + (g >> J.lshift);
    if (S->x == g) atomicAdd(&S->y, d);
    else if (S->z == g) atomicAdd(&S->w, d);
}

__device__ __forceinline__ void set_err(DevState* st, int code)
{
    atomicCAS(&st->err, 0, code);
}

// Adds x to the 64-bit field of job `job` in an array of JobState (field at
// base, records stride_ll long longs apart): one atomic per warp when all of
// its lanes belong to one job (the usual case), one per lane otherwise.
// Every lane of the warp must call it; job < 0 adds nothing.
__device__ __forceinline__ void job_add64(long long x, int job, long long* base, size_t stride_ll)
{
    const unsigned same = __match_any_sync(0xffffffffu, job);
    if (same == 0xffffffffu) {
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0 && x != 0 && job >= 0)
            atomicAdd(reinterpret_cast<unsigned long long*>(base + (size_t)job * stride_ll), (unsigned long long)x);
    } else if (x != 0 && job >= 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(base + (size_t)job * stride_ll), (unsigned long long)x);
    }
}

constexpr size_t kJobStride = sizeof(JobState) / sizeof(long long);

// Per-job 64-bit sums over a kernel's loop: each thread keeps a running
// (job, sum) and flushes it when its job changes -- into a shared-memory
// array of per-job sums when the context has few jobs (sh != nullptr), else
// straight into the job records -- and finish() adds what is left, once per
// warp for one job.  For a single job that is one global atomic per warp per
// launch instead of one per loop iteration.
constexpr int kSmemJobs = 1024;

struct JobAcc {
    int job = -1;
    long long sum = 0;
    long long* sh;      // shared per-job sums or nullptr
    long long* base;    // field of job 0 in the JobState array
    size_t stride;

    __device__ __forceinline__ JobAcc(long long* sh_, long long* base_, size_t stride_)
        : sh(sh_), base(base_), stride(stride_) {}

    __device__ __forceinline__ void flush()
    {
        if (job >= 0 && sum != 0) {
            unsigned long long* dst = reinterpret_cast<unsigned long long*>(sh ? sh + job : base + (size_t)job * stride);
            atomicAdd(dst, (unsigned long long)sum);
        }
        sum = 0;
    }

    __device__ __forceinline__ void add(int j, long long x)
    {
        if (x == 0) return;
        if (j != job) {
            flush();
            job = j;
        }
        sum += x;
    }
};

// Shared per-job sums of a block for contexts of 2..kSmemJobs jobs (dynamic
// shared memory of smem_jobs_bytes(jobs)); nullptr otherwise.  Every thread
// of the block must call it.
__device__ __forceinline__ long long* job_smem_init(int jobs, long long* dyn)
{
    if (jobs < 2 || jobs > kSmemJobs) return nullptr;
    for (int j = threadIdx.x; j < jobs; j += blockDim.x) dyn[j] = 0;
    __syncthreads();
    return dyn;
}

inline size_t smem_jobs_bytes(int jobs)
{
    return (jobs >= 2 && jobs <= kSmemJobs) ? sizeof(long long) * (size_t)jobs : 0;
}

// Adds what the accumulators of the block hold to the job records.  Every
// thread of the block must call it, after its last add().
__device__ __forceinline__ void job_acc_finish(JobAcc& acc, int jobs)
{
    if (acc.sh) {
        acc.flush();
        __syncthreads();
        for (int j = threadIdx.x; j < jobs; j += blockDim.x) {
            const long long x = acc.sh[j];
            if (x != 0) atomicAdd(reinterpret_cast<unsigned long long*>(acc.base + (size_t)j * acc.stride),
                                  (unsigned long long)x);
        }
    } else {
        // lanes that added nothing hold job -1 and sum 0; with one job they
        // join the others so that the warp adds with one atomic
        job_add64(acc.sum, jobs == 1 ? 0 : acc.job, acc.base, acc.stride);
    }
}
static_assert(sizeof(JobState) % sizeof(long long) == 0, "JobState must be a multiple of 8 bytes");

// Count stored under key (0 if absent).  Read-only use during a kernel that
// does not modify the table, so the non-coherent path is allowed.
__device__ __forceinline__ int table_count_ro(const Slot* t, unsigned long long mask, unsigned long long key)
{
    unsigned long long h = hash_key(key) & mask;
    for (unsigned long long p = 0; p <= mask; ++p) {
        ulonglong2 e = __ldg(reinterpret_cast<const ulonglong2*>(t + h));
        if (e.x == key) return (int)(unsigned)(e.y & 0xffffffffull);
        if (e.x == kEmpty) return 0;
        h = (h + 1) & mask;
    }
    return 0;
}

// Slot holding key, or -1 (coherent loads; the key must not be inserted concurrently).
__device__ __forceinline__ long long table_find(const Slot* t, unsigned long long mask, unsigned long long key)
{
    unsigned long long h = hash_key(key) & mask;
    for (unsigned long long p = 0; p <= mask; ++p) {
        unsigned long long k = *reinterpret_cast<const volatile unsigned long long*>(&t[h].key);
        if (k == key) return (long long)h;
        if (k == kEmpty) return -1;
        h = (h + 1) & mask;
    }
    return -1;
}

// Slot holding key, inserting it (count 0, delta 0) if absent.  *inserted is
// set when this call created the slot.  Returns -1 if the table is full.
__device__ __forceinline__ long long table_find_or_insert(Slot* t, unsigned long long mask,
                                                          unsigned long long key, bool* inserted)
{
    *inserted = false;
    unsigned long long h = hash_key(key) & mask;
    for (unsigned long long p = 0; p <= mask; ++p) {
        unsigned long long k = *reinterpret_cast<volatile unsigned long long*>(&t[h].key);
        if (k == key) return (long long)h;
        if (k == kEmpty) {
            unsigned long long old = atomicCAS(&t[h].key, kEmpty, key);
            if (old == kEmpty) { *inserted = true; return (long long)h; }
            if (old == key) return (long long)h;
        }
        h = (h + 1) & mask;
    }
    return -1;
}

// 16-byte compare-and-swap of a whole slot (PTX atom.cas.b128, sm_90 and
// later): returns the slot's previous contents; the swap happened iff they
// equal cmp.
__device__ __forceinline__ ulonglong2 slot_cas(Slot* p, ulonglong2 cmp, ulonglong2 val)
{
    ulonglong2 old;
    asm volatile(
        "{\n\t"
        ".reg .b128 c, v, d;\n\t"
        "mov.b128 c, {%2, %3};\n\t"
        "mov.b128 v, {%4, %5};\n\t"
        "atom.relaxed.gpu.global.cas.b128 d, [%6], c, v;\n\t"
        "mov.b128 {%0, %1}, d;\n\t"
        "}"
        : "=l"(old.x), "=l"(old.y)
        : "l"(cmp.x), "l"(cmp.y), "l"(val.x), "l"(val.y), "l"(p)
        : "memory");
    return old;
}

// 16-byte compare-and-swap of a summary entry (same instruction as slot_cas).
__device__ __forceinline__ ulonglong2 entry_cas(int4* p, ulonglong2 cmp, ulonglong2 val)
{
    return slot_cas(reinterpret_cast<Slot*>(p), cmp, val);
}

// Adds cnt to key's count in a table being built from a cleared state (every
// slot either empty with count 0, or holding a key): a new key is written
// together with its count by one 16-byte CAS; an existing key gets an atomic
// add.  The caller issues the first CAS, at key's home slot h (so that a warp
// can have the first CASes of several keys in flight), and passes its result
// as old; this finishes the insert.  *inserted is set when the insert created
// the slot.  Returns -1 if the key found no slot within `limit` probes.
// mark (0 or 1) goes into the new slot's staged-delta field: the rebuild
// marks the keys whose summary entry is already final (see setup.cu) and
// clears the mark again before any sweep stages deltas.
__device__ __forceinline__ long long table_build_finish(Slot* t, unsigned long long mask, unsigned long long key,
                                                        int cnt, bool* inserted, int mark, unsigned long long limit,
                                                        unsigned long long h, ulonglong2 old)
{
    *inserted = false;
    const ulonglong2 empty = make_ulonglong2(kEmpty, 0ull);
    const ulonglong2 mine =
        make_ulonglong2(key, ((unsigned long long)(unsigned)mark << 32) | (unsigned long long)(unsigned)cnt);
    for (unsigned long long p = 0;;) {
        if (old.x == kEmpty && old.y == 0ull) {
            *inserted = true;
            return (long long)h;
        }
        if (old.x == key) {
            atomicAdd(&t[h].cnt, cnt);
            return (long long)h;
        }
        if (++p > mask || p >= limit) return -1;
        h = (h + 1) & mask;
        old = slot_cas(t + h, empty, mine);
    }
}

// ---- setup.cu ----
// SMs of the current device (queried once per device; 1 if the query fails).
constexpr int kMaxDevices = 64;
int device_sm_count();

// Union assembly: per-job inputs were copied into staging buffers (offsets of
// job j at offstage[vo_j + j ..], n_j + 1 entries; columns job-local at
// col[eo_j ..]); these kernels validate them, build the union offsets, the
// source array and the job of each vertex, and shift the columns to union ids.
struct AssemblyArgs {
    int jobs;
    long long n, nnz;
    const long long* offstage;  // N + J entries
    const long long* eo;        // J + 1: first CSR entry of each job
    const JobInfo* job;
    long long* off;             // N + 1
    int* col;                   // NNZ, job-local on entry, union ids on exit
    int* src;
    int* jid;
    DevState* st;
};
cudaError_t launch_assemble(const AssemblyArgs& a, cudaStream_t s);
// Second half of the assembly (source array, union columns), once the offsets are valid.
cudaError_t launch_assemble_edges(const AssemblyArgs& a, cudaStream_t s);

// Label compaction of all jobs: labels staged partition-major per job (job j's
// k_j x n_j block at lo_j); pjob maps a global partition index (sum of the
// earlier k plus i) to its job, pfirst the job to its first global partition.
struct LabelArgs {
    int jobs;
    long long total;            // sum_j k_j n_j
    const int* labels;          // staged labels
    const long long* lo;        // J + 1: first staged label of each job
    const int* pjob;            // global partition -> job
    const int* pfirst;          // J: first global partition of each job
    const JobInfo* job;
    JobState* js;
    int* G;
    void* lmap;                 // 16-byte slots, lmask + 1 of them
    unsigned long long lmask;
    long long rows;             // entries of G
    DevState* st;
    long long* part_sq;         // per global partition: sum_l |P_il|^2
    double* part_slog;          // per global partition: sum_l |P_il| log |P_il|
};
cudaError_t launch_compact_labels(const LabelArgs& a, cudaStream_t s);
// The same without filling G with -1 first (the caller has set the rows the
// jobs of `a` write, and only those, to -1).
cudaError_t launch_label_kernels(const LabelArgs& a, cudaStream_t s);

cudaError_t launch_init_state(const SweepArgs& a, cudaStream_t s);
// Summary rows of the singleton start ({g_i(v), 1, -1, 0} for cluster v, padding {-1, 0, -1, 0}).
cudaError_t launch_singleton_summaries(const SweepArgs& a, long long rows, cudaStream_t s);
// Sizes from C (ids outside their job set CC_ERR_INVALID).
cudaError_t launch_state_from_ids(const SweepArgs& a, cudaStream_t s);
// Rebuild of the table and summary rows from C into st->new_mask + 1 slots,
// then st->mask = st->new_mask.  conditional: only if st->rebuild is set.
// eval: in a heavy sweep, also add the table part of F' to each job's recompute.
cudaError_t launch_table_rebuild(const SweepArgs& a, long long rows, bool conditional, cudaStream_t s,
                                 bool eval = false);
// F of every job from scratch into js[j].recompute (without sum_ij |P_ij|^2).
cudaError_t launch_objective_recompute(const SweepArgs& a, cudaStream_t s);

// ---- metrics.cu ----
// Sums for the partition distances of every job's consensus against each of
// its input partitions, from a freshly rebuilt table (its summary rows hold
// each (cluster, partition)'s largest overlap).  Per global partition P (job
// j's partition i is P = pfirst[j] + i): sq[P] = sum n(c,i,l)^2, slog[P] =
// sum n log n, sjc[P] = sum over clusters c of max_l n(c,i,l), sjl[P] = sum
// over classes l of max_c n(c,i,l); per job: csq[j] = sum |c|^2, cslog[j] =
// sum |c| log |c|.  lmax: one int per label id of every job (job j's ids start
// at lbase[j]); all outputs zeroed by the caller.
struct MetricsArgs {
    const int* pfirst;
    const long long* lbase;
    long long nlabels;      // entries of lmax
    int* lmax;
    long long* sq;
    double* slog;
    long long* sjc;
    long long* sjl;
    long long* csq;
    double* cslog;
};
cudaError_t launch_metrics(const SweepArgs& a, const MetricsArgs& m, int parts, cudaStream_t s);
// C of job j's n vertices := its input partition i (cluster id = least vertex of the class).
cudaError_t launch_ids_from_partition(const SweepArgs& a, long long n, int j, int i, cudaStream_t s);

// Greedy colouring of every job's graph in decreasing splitmix64 priority of
// job-local vertex ids (Jones-Plassmann rounds), then the vertices and CSR
// entries listed class by class; *classes receives the number of classes.
// colour, vlist (n), eidx (nnz), voff / eoff (n + 2 entries) are allocated by
// the caller; cnt (8 (n + 2) bytes) is scratch.
struct ColourArgs {
    long long n, nnz;
    const long long* off;
    const int* col;
    const int* jid;
    const JobInfo* job;
    int* colour;
    int* vlist;
    int* voff;
    int* eidx;
    long long* eoff;
    long long* cnt;
    int* flag;              // one int of scratch
};
cudaError_t launch_colouring(const ColourArgs& a, int* classes, cudaStream_t s);

// ---- api.cu ----
// Message reported by cc_last_error(NULL) in this thread.
void set_thread_error(const std::string& msg);

// ---- sweep.cu ----
cudaError_t launch_run_begin(const SweepArgs& a, int limit, cudaStream_t s);
// One sweep of every job; prop0/prop1 (may be null) are recorded around the
// proposal kernels.  With a body stream (while s is being captured into a
// graph), the heavy path, its rollback, the light path and the end-of-sweep
// rebuild become IF regions of the graph, each behind a one-thread gate
// kernel, so a sweep launches only the regions it needs.
constexpr int kKernelsPerRebuild = 9;
// regions: heavy path (mark, apply, rebuild), its second rebuild attempt,
// heavy evaluation (eval, decide), rollback (undo, rebuild), light path
// (stage, eval, decide), end-of-sweep rebuild
constexpr int kKernelsInRegions = (2 + kKernelsPerRebuild) + kKernelsPerRebuild + 2 + (1 + kKernelsPerRebuild) + 3 +
                                  kKernelsPerRebuild;
constexpr int kKernelsPerSweep = 11 + kKernelsInRegions;  // kernels of a sweep without regions
constexpr int kGatesPerSweep = 6;
// kernels of a sweep graph outside its regions (gates included); the kernels
// of the regions that run are counted on the device (DevState.region_launches)
constexpr int kKernelsOutsideRegions = kKernelsPerSweep + kGatesPerSweep - kKernelsInRegions;
cudaError_t launch_sweep(const SweepArgs& a, long long rows, int grid, cudaStream_t s, cudaEvent_t prop0,
                         cudaEvent_t prop1, cudaStream_t body = nullptr);
cudaError_t prepare_propose(int* blocks_per_sm);
// Adds to the graph being captured on s a WHILE node whose body (captured on
// `loop`, with the sweep's regions on `body`) is one sweep followed by a gate
// that repeats it until the run stops, fails or has run `budget` bodies: a
// whole run as one graph launch.
cudaError_t capture_run_loop(const SweepArgs& a, long long rows, int grid, cudaStream_t s, cudaStream_t loop,
                             cudaStream_t body, int budget);
// The proposal step's scoring kernels alone (own-cluster sums, candidate
// bids) on the current state, for timing; they write only aown, act (the
// same values on the same state) and the bids, which launch_clear_bids
// empties again.  Nothing else of the state changes.
cudaError_t launch_propose_probe(const SweepArgs& a, int grid, cudaStream_t s);
cudaError_t launch_clear_bids(const SweepArgs& a, int grid, cudaStream_t s);

}  // namespace ccg
