// Internal declarations shared by the CUDA translation units of libcc.so.
//
// Device data layout (one consensus job):
//   off   int64[n+1]   CSR row offsets            col  int32[nnz]  neighbours
//   G     int32[n][kp] compacted label ids, vertex-major, kp = k rounded up to 4 so
//                      that each row is 16-byte aligned; g = (i << s) | rep where rep
//                      is the least vertex carrying that label in partition i and
//                      2^s >= n, so g identifies (partition, label), i = g >> s and
//                      g < k 2^s < 2 k n.  Padding = -1.
//   summ  int4[n][kp]  per (cluster x, partition i): {d, m, m2, 0} with d the label id
//                      that was most frequent in x at the last table rebuild, m the
//                      exact current count of d in x (kept by every commit) and m2 an
//                      upper bound on the count of every other label of partition i
//                      in x (raised by commits, recomputed at rebuilds).
//   C     int32[n]     cluster id of each vertex (founding-vertex ids)
//   size  int32[n]     cluster sizes, indexed by cluster id
//   table Slot[cap]    the contingency counts n(c, i, l) as an open-addressing
//                      hash with linear probing, key = c << 32 | g.  The buffer holds
//                      2^p >= 3 k n slots; only an active prefix of 2^q slots is used
//                      (st->mask = 2^q - 1), grown before a sweep stages its moves and
//                      shrunk when few keys are live, so that the probes of late
//                      sweeps stay in L2.
#pragma once

#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "cc.h"

namespace ccg {

constexpr unsigned long long kEmpty = ~0ull;
constexpr int kWarpsPerBlock = 8;
constexpr int kBlock = kWarpsPerBlock * 32;
constexpr int kTile = 256;  // vertices claimed at once by a block of the proposal kernel

// One contingency entry: the (cluster, label id) key, its count and the
// delta staged by the current sweep.  16 bytes, read as one vector load.
struct __align__(16) Slot {
    unsigned long long key;
    int cnt;
    int dlt;
};

// Device-resident control block of a context.
struct DevState {
    unsigned long long nprop;    // |P| of the current sweep
    unsigned long long np1;      // |P1|
    long long dF;                // staged objective change
    long long dF_p1;             // dF of P1 as evaluated
    long long F;                 // current objective
    unsigned long long moves;    // moves committed in the current sweep
    unsigned long long used;     // occupied table slots
    long long live;              // keys with a non-zero count
    unsigned long long tile_ctr; // next vertex tile of the proposal kernel
    unsigned long long mask;     // active table capacity - 1 (a power of two minus one)
    unsigned long long new_mask; // capacity - 1 of a pending rebuild
    long long partition_sq;      // sum_i sum_j |P_ij|^2
    long long recompute;         // output of the full objective reduction
    int mode;                    // 0 nothing to commit, 1 commit P1, 2 matching
    int overflow;                // 1: the table ran short during this sweep (nothing committed)
    int abort;                   // 1: the pending rebuild follows an abandoned sweep
    int retries;                 // sweeps abandoned and retried in a larger table
    int heavy;                   // 1: this sweep evaluates P1 by a rebuild (see sweep.cu)
    int rollback;                // 1: the heavy sweep's P1 was rejected and is being undone
    int tvalid;                  // 1: the table holds the counts of the current C
    int rebuilds;                // table rebuilds since creation
    int skip;                    // 1: this sweep does nothing (the run has stopped)
    int stop;                    // 1: the run has stopped
    int rebuild;                 // 1: a table rebuild is pending
    int err;                     // cc_status of a device-side failure (first one wins)
    int sweeps;                  // sweeps recorded since creation / reset
    int run_sweeps;              // sweeps in the current run
    int run_limit;               // sweep limit of the current run
};

// Arguments of the sweep kernels (passed by value).
struct SweepArgs {
    int n, k, kp;
    long long nnz;
    const long long* off;
    const int* col;
    const int* src;             // source vertex of each CSR entry (nnz)
    const int* G;
    int* C;
    int* size;
    int* dsize;                 // staged size deltas
    unsigned long long* best;   // bids: per vertex in the proposal step, per cluster in the matching
    int* aown;                  // A_a of each vertex for the current sweep
    Slot* table;
    int4* summ;                  // per-cluster label summaries (see above)
    int lshift;                  // s: label id g = (i << s) | rep
    int sweep_mode;              // 0 automatic, 1 always staged deltas, 2 always rebuild
    unsigned long long mask_max; // allocated capacity - 1; the active capacity is st->mask + 1
    unsigned long long cap_min;  // smallest active capacity
    int* pv;                    // proposal list: vertex,
    int* pa;                    //   source cluster,
    int* pb;                    //   target cluster,
    int* pg;                    //   gain dD
    unsigned char* pflag;       //   1 if kept by the singleton guard
    unsigned int* pslot;        //   table slots of (a, g_i(v)) and (b, g_i(v)), 2 per (j, i)
    int* members;               // rebuild scratch: vertices listed cluster by cluster (n)
    int* cursor;                // rebuild scratch: next free position of each cluster (n)
    int* bsum;                  // rebuild scratch: per-block sums of the size scan (n / 1024 + 1)
    DevState* st;
    cc_sweep_info* hist;
    int hist_cap;
};

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
// 2^32 slots (at most 4 k n rounded up, with 3 k n < 2^31).
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

// Keeps the summary row of the slot's (cluster, partition) valid after its
// count changed by d to newc: the count of the row's label is exact, the
// bound on the other labels only rises.
__device__ __forceinline__ void summ_update(int4* summ, int kp, int lshift, unsigned long long key, int d, int newc)
{
    const int x = (int)(key >> 32), g = (int)(unsigned)(key & 0xffffffffull);
    int4* S = summ + (long long)x * kp + (g >> lshift);
    if (S->x == g) atomicAdd(&S->y, d);
    else if (d > 0) atomicMax(&S->z, newc);
}

__device__ __forceinline__ void set_err(DevState* st, int code)
{
    atomicCAS(&st->err, 0, code);
}

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

// ---- launch wrappers (setup.cu) ----
cudaError_t launch_validate(int n, long long nnz, const long long* off, const int* col, DevState* st,
                            cudaStream_t s);
cudaError_t launch_fill_src(int n, const long long* off, int* src, cudaStream_t s);
cudaError_t launch_compact_labels(int n, int k, int kp, int lshift, const int* labels, int* G, void* lmap,
                                  unsigned long long lmask, DevState* st, cudaStream_t s);
cudaError_t launch_init_state(const SweepArgs& a, cudaStream_t s);
// Summary rows of the singleton start ({g_i(v), 1, 0} for cluster v).
cudaError_t launch_singleton_summaries(const SweepArgs& a, cudaStream_t s);
cudaError_t launch_state_from_ids(const SweepArgs& a, cudaStream_t s);
// Rebuild of the table from C into st->new_mask + 1 slots, then st->mask = st->new_mask.
// conditional: only if st->rebuild is set (decided on the device).
cudaError_t launch_table_rebuild(const SweepArgs& a, bool conditional, cudaStream_t s);
cudaError_t launch_objective_recompute(const SweepArgs& a, cudaStream_t s);

// ---- api.cu ----
// Message reported by cc_last_error(NULL) in this thread.
void set_thread_error(const std::string& msg);

// ---- launch wrappers (sweep.cu) ----
cudaError_t launch_run_begin(DevState* st, int limit, cudaStream_t s);
// One sweep (13 kernels); prop0/prop1 (may be null) are recorded around the proposal kernel.
constexpr int kKernelsPerRebuild = 11;
constexpr int kKernelsPerSweep = 18 + 3 * kKernelsPerRebuild;
cudaError_t launch_sweep(const SweepArgs& a, int grid, cudaStream_t s, cudaEvent_t prop0, cudaEvent_t prop1);
cudaError_t prepare_propose(int kp, int* blocks_per_sm);

}  // namespace ccg
