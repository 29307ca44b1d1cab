// Setup of the jobs of a context (The algorithm: Initialization) and the
// table maintenance kernels: union assembly with input validation, per-job
// label compaction into the vertex-major membership matrix, the singleton
// state, the contingency hash rebuild with its summary rows, and the
// from-scratch objective used for checks.
#include <algorithm>
#include <atomic>
#include <climits>
#include <vector>

#include "cc_internal.cuh"

namespace ccg {

int device_sm_count()
{
    static std::atomic<int> cache[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
    if (dev < kMaxDevices) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 1;
    if (dev < kMaxDevices) cache[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

namespace {

constexpr int kSetupBlock = 256;

// Grid for grid-stride kernels: one block per kSetupBlock items, at most 16
// resident blocks per SM of the current device.
inline int grid_for(long long work, int per_block = kSetupBlock)
{
    const long long max_blocks = 16LL * device_sm_count();
    long long b = (work + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

// (global partition, raw label) -> least job-local vertex carrying it, and the class size.
struct __align__(16) LSlot {
    unsigned long long key;
    int rep;
    int cnt;
};

// Largest index i with key[i] <= x among key[0..count) (key[0] <= x assumed).
__device__ __forceinline__ int upper_index(const long long* key, int count, long long x)
{
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (key[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int job_of_vertex(const JobInfo* job, int jobs, long long v)
{
    int lo = 0, hi = jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (job[mid].vo <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---- union assembly -------------------------------------------------------

__global__ void k_fill_jid(AssemblyArgs a)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += stride)
        a.jid[v] = job_of_vertex(a.job, a.jobs, v);
}

// off[v] = eo_j + (job-local offset); checks each job's offsets start at 0, do
// not decrease and end at its nnz.
__global__ void k_assemble_off(AssemblyArgs a)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += stride) {
        const int j = a.jid[v];
        const JobInfo J = a.job[j];
        const long long vl = v - J.vo;
        const long long* o = a.offstage + J.vo + j;  // the job's n + 1 offsets
        const long long here = o[vl], next = o[vl + 1];
        bool bad = next < here;
        if (vl == 0 && here != 0) bad = true;
        if (vl == J.n - 1 && next != a.eo[j + 1] - a.eo[j]) bad = true;
        if (bad) atomicCAS(&a.st->err, 0, (int)CC_ERR_INVALID);
        a.off[v] = a.eo[j] + here;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.off[a.n] = a.nnz;
}

__global__ void k_fill_src(AssemblyArgs a)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += stride)
        for (long long e = a.off[v]; e < a.off[v + 1] && e < a.nnz; ++e) a.src[e] = (int)v;
}

__global__ void k_assemble_col(AssemblyArgs a)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < a.nnz; e += stride) {
        const JobInfo J = a.job[a.jid[a.src[e]]];
        const int c = a.col[e];
        if (c < 0 || c >= J.n) {
            atomicCAS(&a.st->err, 0, (int)CC_ERR_INVALID);
            a.col[e] = (int)J.vo;
        } else {
            a.col[e] = (int)(J.vo + c);
        }
    }
}

// ---- label compaction -----------------------------------------------------

__global__ void k_lmap_clear(LSlot* m, unsigned long long cap)
{
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; s < cap; s += stride) {
        m[s].key = kEmpty;
        m[s].rep = INT_MAX;
        m[s].cnt = 0;
    }
}

__device__ __forceinline__ long long lmap_slot(LSlot* m, unsigned long long mask, unsigned long long key, bool insert)
{
    unsigned long long h = mix64(key) & mask;
    for (unsigned long long p = 0; p <= mask; ++p) {
        unsigned long long k = *reinterpret_cast<volatile unsigned long long*>(&m[h].key);
        if (k == key) return (long long)h;
        if (k == kEmpty) {
            if (!insert) return -1;
            unsigned long long old = atomicCAS(&m[h].key, kEmpty, key);
            if (old == kEmpty || old == key) return (long long)h;
        }
        h = (h + 1) & mask;
    }
    return -1;
}

// Entry t of the staged labels: its job, partition and job-local vertex.
__device__ __forceinline__ void label_entry(const LabelArgs& a, long long t, int& j, int& i, long long& vl)
{
    j = upper_index(a.lo, a.jobs, t);
    const long long tl = t - a.lo[j];
    const long long n = a.job[j].n;
    i = (int)(tl / n);
    vl = tl - (long long)i * n;
}

__global__ void k_label_insert(LabelArgs a)
{
    LSlot* m = static_cast<LSlot*>(a.lmap);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < a.total; t += stride) {
        int j, i;
        long long vl;
        label_entry(a, t, j, i, vl);
        const unsigned long long key = ((unsigned long long)(unsigned)(a.pfirst[j] + i) << 32) | (unsigned)a.labels[t];
        const long long s = lmap_slot(m, a.lmask, key, true);
        if (s < 0) { set_err(a.st, CC_ERR_TABLE_FULL); continue; }
        atomicMin(&m[s].rep, (int)vl);
        atomicAdd(&m[s].cnt, 1);
    }
}

// G[row(v) + i] = (i << s_j) | rep(i, label); G was filled with -1 before, so
// the padding entries keep -1.
__global__ void k_label_assign(LabelArgs a)
{
    const LSlot* m = static_cast<const LSlot*>(a.lmap);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < a.total; t += stride) {
        int j, i;
        long long vl;
        label_entry(a, t, j, i, vl);
        const JobInfo J = a.job[j];
        const unsigned long long key = ((unsigned long long)(unsigned)(a.pfirst[j] + i) << 32) | (unsigned)a.labels[t];
        const long long s = lmap_slot(const_cast<LSlot*>(m), a.lmask, key, false);
        if (s < 0) {
            set_err(a.st, CC_ERR_INVALID);
            continue;
        }
        a.G[J.go + vl * J.kp + i] = (i << J.lshift) | m[s].rep;
    }
}

// sum_i sum_j |P_ij|^2 of every job.
__global__ void k_label_sumsq(LabelArgs a, unsigned long long cap)
{
    extern __shared__ long long dyn_jobs[];
    const LSlot* m = static_cast<const LSlot*>(a.lmap);
    JobAcc acc(job_smem_init(a.jobs, dyn_jobs), &a.js[0].partition_sq, kJobStride);
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; s < cap; s += stride) {
        if (m[s].key == kEmpty) continue;
        const long long c = m[s].cnt;
        const int P = (int)(m[s].key >> 32);
        acc.add(a.pjob[P], c * c);
        atomicAdd(reinterpret_cast<unsigned long long*>(a.part_sq + P), (unsigned long long)(c * c));
        atomicAdd(a.part_slog + P, (double)c * log((double)c));
    }
    job_acc_finish(acc, a.jobs);
}

// ---- state ----------------------------------------------------------------

__global__ void k_init_state(SweepArgs a)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += stride) {
        a.C[v] = (int)v;
        a.size[v] = 1;
        a.dsize[v] = 0;
        a.best[v] = kEmpty;
        a.chg[v] = -2;  // stamps start at 0: never "the previous sweep"
        a.prev[v] = kEmpty;
        a.act[v] = 1;
    }
}

__global__ void k_summ_singletons(SweepArgs a, long long rows)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += stride) {
        const int g = a.G[r];
        a.summ[r] = make_int4(g, g >= 0 ? 1 : 0, -1, 0);
    }
}

__global__ void k_sizes_zero(SweepArgs a)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += stride) {
        a.size[v] = 0;
        a.dsize[v] = 0;
        a.best[v] = kEmpty;
    }
}

// Sizes from a given consensus; an id outside its vertex's job sets an error.
__global__ void k_count_sizes(SweepArgs a)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += stride) {
        const JobInfo& J = a.job[a.jid[v]];
        const long long c = a.C[v];
        if (c < J.vo || c >= J.vo + J.n) set_err(a.st, CC_ERR_INVALID);
        else atomicAdd(&a.size[c], 1);
    }
}

// ---- table rebuild ------------------------------------------------------
// The table is rebuilt from C alone: clear the capacity being built, list the
// vertices cluster by cluster (counting sort: an exclusive scan of the sizes
// gives each cluster's first position), then insert the keys with partitions
// innermost per member, so that the 32 lanes of a warp hold consecutive
// members of (mostly) one cluster for one partition: equal keys are merged
// with __match_any_sync and added with one atomic.  The summary rows follow
// from the rebuilt counts.  All kernels are skipped unless a rebuild is
// pending (conditional) and run unconditionally otherwise.

__device__ __forceinline__ bool rebuild_off(const DevState* st, int conditional)
{
    return conditional && (!st->rebuild || st->err);
}

// Clears the slots of the capacity being built (st->new_mask + 1 of them),
// the summary rows, the occupied-slot counter, and the staged size deltas
// after an abandoned sweep.  Summary rows: those of the live clusters (a warp
// per 32 cluster ids, the lanes across each live row), which are the rows the
// rebuild fills and the sweeps read.  The row of a dead cluster is never read
// again, since no move enters an empty cluster, except with empty_moves (a
// vertex may found a cluster under its own, possibly dead, id); then, and
// when the table did not hold the counts of C before (a new start), every row
// is cleared.
__global__ void k_table_clear(SweepArgs a, long long rows, int conditional)
{
    DevState* st = a.st;
    if (rebuild_off(st, conditional)) return;
    const unsigned long long cap = st->new_mask + 1;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long t0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (unsigned long long s = t0; s < cap; s += stride)
        reinterpret_cast<ulonglong2*>(a.table)[s] = make_ulonglong2(kEmpty, 0ull);
    const int4 none = make_int4(-1, 0, -1, 0);
    if (a.empty_moves || !st->tvalid) {
        for (unsigned long long r = t0; r < (unsigned long long)rows; r += stride) a.summ[r] = none;
    } else {
        const int lane = threadIdx.x & 31;
        for (unsigned long long x0 = t0 - lane; x0 < (unsigned long long)a.n; x0 += stride) {
            const unsigned long long x = x0 + lane;
            unsigned live = __ballot_sync(0xffffffffu, x < (unsigned long long)a.n && a.size[x] > 0);
            while (live) {
                const long long xx = (long long)x0 + __ffs(live) - 1;
                live &= live - 1;
                const JobInfo& J = a.job[a.jid[xx]];
                int4* row = a.summ + row_of(J, xx);
                for (int q = lane; q < J.kp; q += 32) row[q] = none;
            }
        }
    }
    if (st->abort)
        for (unsigned long long v = t0; v < (unsigned long long)a.n; v += stride) a.dsize[v] = 0;
    if (t0 == 0) st->used = 0;
}

__device__ __forceinline__ int warp_incl_scan(int x, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Block sums of size[] over blocks of 1024 entries.
__global__ void __launch_bounds__(1024) k_scan_blocks(SweepArgs a, int conditional)
{
    if (rebuild_off(a.st, conditional)) return;
    __shared__ int wsum[32];
    const long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = i < a.n ? a.size[i] : 0;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int y = wsum[lane];
        for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
        if (lane == 0) a.bsum[blockIdx.x] = y;
    }
}

// Exclusive scan of the nb block sums in place (one block, 1024 threads, each
// owning a contiguous run).
__global__ void __launch_bounds__(1024) k_scan_sums(SweepArgs a, int nb, int conditional)
{
    if (rebuild_off(a.st, conditional)) return;
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int per = (nb + 1023) / 1024;
    const int lo = threadIdx.x * per, hi = min(nb, lo + per);
    int sum = 0;
    for (int b = lo; b < hi; ++b) sum += a.bsum[b];
    int x = warp_incl_scan(sum, lane);
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) wsum[lane] = warp_incl_scan(wsum[lane], lane);
    __syncthreads();
    int run = x - sum + (w > 0 ? wsum[w - 1] : 0);
    for (int b = lo; b < hi; ++b) {
        const int y = a.bsum[b];
        a.bsum[b] = run;
        run += y;
    }
}

// cursor[c] = exclusive prefix of size[] (the first position of cluster c).
__global__ void __launch_bounds__(1024) k_scan_write(SweepArgs a, int conditional)
{
    if (rebuild_off(a.st, conditional)) return;
    __shared__ int wsum[32];
    const long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int v = i < a.n ? a.size[i] : 0;
    int x = warp_incl_scan(v, lane);
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) wsum[lane] = warp_incl_scan(wsum[lane], lane);
    __syncthreads();
    if (i < a.n) a.cursor[i] = a.bsum[blockIdx.x] + x - v + (w > 0 ? wsum[w - 1] : 0);
}

__global__ void k_members_scatter(SweepArgs a, int conditional)
{
    if (rebuild_off(a.st, conditional)) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += stride) {
        const int pos = atomicAdd(&a.cursor[a.C[v]], 1);
        if (pos < a.n) a.members[pos] = (int)v;
        else set_err(a.st, CC_ERR_INVALID);  // sizes inconsistent with C
    }
}

// Largest 64-bit value over the lanes of a contiguous lane segment [lane,
// end) of the warp, left in the segment's first lane (every lane must call it).
__device__ __forceinline__ unsigned long long segment_max(unsigned long long x, int lane, int end)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_down_sync(0xffffffffu, x, o);
        if (lane + o < end && y > x) x = y;
    }
    return x;
}

// Inserts every member's keys (partitions innermost, equal keys of a warp
// merged with __match_any_sync and added once).  Members are listed cluster
// by cluster, so a cluster whose members all lie in one warp's 32 entries
// gets its exact counts inside that warp: the warp then writes the cluster's
// summary entries itself (the two most frequent labels, ties to the larger
// id, as the table scan would rank them), adds its keys' -2 n^2 to the job's
// F' in a heavy sweep (eval), and marks those keys so that the scan skips
// them.  Keys of clusters spread over several warps are left to the scan.
// A tight attempt (see k_build_check) gives every insert kTightProbes probes;
// an insert that finds no slot within them flags the attempt as failed, and
// the warps stop inserting.
constexpr unsigned long long kTightProbes = 256;

__global__ void __launch_bounds__(kSetupBlock, 4) k_table_build(SweepArgs a, int conditional, int eval)
{
    extern __shared__ long long dyn_jobs[];
    DevState* st = a.st;
    if (rebuild_off(st, conditional)) return;
    __shared__ unsigned long long s_used;
    if (threadIdx.x == 0) s_used = 0;
    // tight attempts are made only by the heavy sweep's rebuild inside a
    // sweep graph; a rebuild the host asks for is never one
    const bool tight = conditional && st->tight != 0;
    const unsigned long long limit = tight ? kTightProbes : ~0ull;
    const bool ev = eval && st->heavy;
    JobAcc acc(ev ? job_smem_init(a.jobs, dyn_jobs) : nullptr, &a.js[0].recompute, kJobStride);
    __syncthreads();
    const unsigned long long mask = st->new_mask;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    unsigned long long used = 0;  // slots this warp created (lane 0 counts)
    for (long long base = (long long)blockIdx.x * blockDim.x; base < a.n; base += stride) {
        if (tight && __any_sync(0xffffffffu, *reinterpret_cast<volatile int*>(&st->build_fail) != 0)) break;
        const long long m = base + threadIdx.x;
        const long long wb = m - lane;  // first member of this warp's window
        const bool valid = m < a.n;
        int v = 0, c = 0, k = 0, job = 0, seg_end = lane + 1;
        bool whole = false;
        const int* row = a.G;
        int4* S = a.summ;
        if (valid) {
            v = a.members[m];
            c = a.C[v];
            job = a.jid[v];
            const JobInfo& J = a.job[job];
            k = J.k;
            row = a.G + row_of(J, v);
            // after the scatter, cursor[c] is one past the cluster's last member
            const long long end = a.cursor[c], first = end - a.size[c];
            whole = first >= wb && end <= wb + 32;
            if (whole) seg_end = (int)(end - wb);
            S = a.summ + row_of(J, c);
        }
        const int hl = whole ? (int)((long long)a.cursor[c] - a.size[c] - wb) : lane;  // the cluster's first lane
        const bool head = whole && hl == lane;
        // the warp's whole clusters need the summary maxima; a warp without
        // any skips them
        const bool any_whole = __any_sync(0xffffffffu, whole);
        const int4* G4 = reinterpret_cast<const int4*>(row);
        const ulonglong2 empty = make_ulonglong2(kEmpty, 0ull);
        const unsigned long long mark = whole ? (1ull << 32) : 0ull;
        // four partitions at a time: one quad of the label row, and the four
        // keys' first CASes issued before any result is used
        for (int i0 = 0; i0 < a.kmax; i0 += 4) {
            int4 g4 = make_int4(0, 0, 0, 0);
            if (valid && i0 < k) g4 = __ldg(G4 + (i0 >> 2));
            const int gq[4] = {g4.x, g4.y, g4.z, g4.w};
            unsigned long long key[4], h[4];
            int cnt[4];
            bool lead[4];
            ulonglong2 old[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const bool on = valid && i0 + b < k;
                key[b] = on ? ckey(c, gq[b]) : kEmpty;
                const unsigned same = __match_any_sync(0xffffffffu, key[b]);
                cnt[b] = __popc(same);
                lead[b] = on && (__ffs(same) - 1) == lane;
                h[b] = hash_key(key[b]) & mask;
            }
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if (lead[b]) old[b] = slot_cas(a.table + h[b], empty, make_ulonglong2(key[b], mark | (unsigned)cnt[b]));
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                bool ins = false;
                if (lead[b]) {
                    if (table_build_finish(a.table, mask, key[b], cnt[b], &ins, whole ? 1 : 0, limit, h[b], old[b]) <
                        0) {
                        if (tight) st->build_fail = 1;
                        else set_err(st, CC_ERR_TABLE_FULL);
                    }
                    if (ev && whole) acc.add(job, -2LL * cnt[b] * cnt[b]);
                }
                used += __popc(__ballot_sync(0xffffffffu, ins));
            }
            if (!any_whole) continue;
            // summary entries of the whole clusters: the two largest (count, label)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const bool on = valid && i0 + b < k;
                const unsigned long long mine =
                    (whole && on) ? ((unsigned long long)(unsigned)cnt[b] << 32) | (unsigned)gq[b] : 0ull;
                const unsigned long long top1 = segment_max(mine, lane, seg_end);
                const unsigned long long t1 = __shfl_sync(0xffffffffu, top1, hl);
                const unsigned long long other = (mine != 0 && (unsigned)mine != (unsigned)t1) ? mine : 0ull;
                const unsigned long long top2 = segment_max(other, lane, seg_end);
                if (head && on) {
                    const int d2 = top2 ? (int)(unsigned)top2 : -1, m2 = (int)(top2 >> 32);
                    S[i0 + b] = make_int4((int)(unsigned)top1, (int)(top1 >> 32), d2, m2);
                }
            }
        }
    }
    // one add per block: st->used is a single word that every block updates
    if (lane == 0 && used) atomicAdd(&s_used, used);
    if (ev) job_acc_finish(acc, a.jobs);
    __syncthreads();
    if (threadIdx.x == 0 && s_used) atomicAdd(&st->used, s_used);
}

// Summary rows of the rebuilt table for the keys the build left unmarked
// (clusters spread over several warps).  Each half of a row entry reads as
// one unsigned 64-bit value (count << 32 | label id); every such slot offers
// its (count, label) to the entry, which keeps the two largest by a 16-byte
// compare-and-swap (ties to the larger id; cleared entries hold count 0 and
// label -1, below any real key).  Content does not depend on the order of
// the offers.  Marked slots only get their mark cleared.
// With eval set (the first rebuild of a heavy sweep) this pass also adds
// -2 sum n^2 over the unmarked keys to each job's recompute (the table part
// of F'; the build added the marked ones).
__global__ void k_summ_top(SweepArgs a, int conditional, int eval)
{
    extern __shared__ long long dyn_jobs[];
    DevState* st = a.st;
    if (rebuild_off(st, conditional) || st->again) return;
    const bool ev = eval && st->heavy;
    JobAcc acc(ev ? job_smem_init(a.jobs, dyn_jobs) : nullptr, &a.js[0].recompute, kJobStride);
    const unsigned long long cap = st->new_mask + 1;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; s < cap; s += stride) {
        const ulonglong2 e = reinterpret_cast<const ulonglong2*>(a.table)[s];
        const int cnt = (int)(unsigned)(e.y & 0xffffffffull);
        if (e.x == kEmpty || cnt <= 0) continue;
        if ((e.y >> 32) != 0) {
            a.table[s].dlt = 0;  // summary and F' part done by the build
            continue;
        }
        const int x = (int)(e.x >> 32), g = (int)(unsigned)(e.x & 0xffffffffull);
        const int job = a.jid[x];
        const JobInfo& J = a.job[job];
        int4* E = a.summ + row_of(J, x) + (g >> J.lshift);
        const unsigned long long kn = ((unsigned long long)(unsigned)cnt << 32) | (unsigned)g;
        const volatile unsigned long long* Ev = reinterpret_cast<const volatile unsigned long long*>(E);
        ulonglong2 cur = make_ulonglong2(Ev[0], Ev[1]);
        // lock-free: every failed swap means another offer went in; bounded
        // all the same
        for (int tries = 0; kn > cur.y; ++tries) {
            if (tries >= (1 << 20)) {
                set_err(st, CC_ERR_INVALID);
                break;
            }
            const ulonglong2 nv = kn > cur.x ? make_ulonglong2(kn, cur.x) : make_ulonglong2(cur.x, kn);
            const ulonglong2 old = entry_cas(E, cur, nv);
            if (old.x == cur.x && old.y == cur.y) break;
            cur = old;
        }
        if (ev) acc.add(job, -2LL * cnt * cnt);
    }
    if (ev) job_acc_finish(acc, a.jobs);
}

// Check of a tight attempt, after its build: the table must have taken every
// key within the probe limit, at load <= 1/2, with room left below the fill
// limit for the new keys of a light sweep (at most 2 x sum_j k_j n_j / 8).
// Otherwise the attempt is dropped (its part of F' is cleared; the summary
// pass and the done step skip it) and the rebuild runs again at the capacity
// that holds every key the sweep can create.  One block.
__global__ void k_build_check(SweepArgs a, int conditional)
{
    DevState* st = a.st;
    if (rebuild_off(st, conditional)) return;
    __shared__ int fail;
    if (threadIdx.x == 0) {
        fail = 0;
        if (conditional && st->tight) {
            const unsigned long long cap = st->new_mask + 1, fill = cap - (cap >> 3);
            const unsigned long long room = 2 * ((a.keys + 7) / 8);
            fail = st->build_fail || st->used > cap / 2 || st->used + room > fill || a.tight_mode == 2;
        }
    }
    __syncthreads();
    if (fail)
        for (int j = threadIdx.x; j < a.jobs; j += blockDim.x) a.js[j].recompute = 0;
    if (threadIdx.x == 0) {
        if (fail) st->new_mask = st->safe_mask;
        st->again = fail;
        st->tight = 0;
        st->build_fail = 0;
    }
}

__global__ void k_table_done(DevState* st, int conditional)
{
    if (rebuild_off(st, conditional) || st->again) return;
    st->live = (long long)st->used;
    st->mask = st->new_mask;
    st->rebuild = 0;
    st->abort = 0;
    st->rebuilds += 1;
    st->tvalid = 1;
}

// F of every job without sum_ij |P_ij|^2: k sum_c s_c^2 - 2 sum_keys n^2.
__global__ void k_objective_recompute(SweepArgs a)
{
    extern __shared__ long long dyn_jobs[];
    JobAcc acc(job_smem_init(a.jobs, dyn_jobs), &a.js[0].recompute, kJobStride);
    const unsigned long long mask = a.st->mask;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long t0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (unsigned long long t = t0; t < (unsigned long long)a.n; t += stride) {
        const long long s = a.size[t];
        if (s > 0) {
            const int j = a.jid[t];
            acc.add(j, (long long)a.job[j].k * s * s);
        }
    }
    for (unsigned long long t = t0; t <= mask; t += stride) {
        const ulonglong2 e = reinterpret_cast<const ulonglong2*>(a.table)[t];
        const long long c = (int)(unsigned)(e.y & 0xffffffffull);
        if (e.x != kEmpty && c != 0) acc.add(a.jid[(int)(e.x >> 32)], -2 * c * c);
    }
    job_acc_finish(acc, a.jobs);
}

__global__ void k_zero_recompute(SweepArgs a)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < a.jobs; j += gridDim.x * blockDim.x)
        a.js[j].recompute = 0;
}

// ---- colouring (colour_batched) ------------------------------------------
// Priority of a job-local vertex id: the first output of splitmix64 (Steele,
// Lea and Flood) seeded with it; a bijection, so priorities are distinct.
__device__ __forceinline__ unsigned long long colour_priority(unsigned long long v)
{
    unsigned long long z = v + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_colour_init(ColourArgs a)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += stride) a.colour[v] = -1;
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.flag = 0;
}

// One Jones-Plassmann round: an uncoloured vertex whose higher-priority
// neighbours are all coloured takes the least colour none of them has, which
// is what the greedy colouring in decreasing priority gives it.  A colour, once
// written, is final, so a vertex that sees a neighbour coloured in this same
// round sees its final colour.  *flag counts the vertices left uncoloured.
__global__ void k_colour_round(ColourArgs a)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const volatile int* colour = a.colour;
    int left = 0;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += stride) {
        if (colour[v] >= 0) continue;
        const long long vo = a.job[a.jid[v]].vo;
        const unsigned long long pv = colour_priority((unsigned long long)(v - vo));
        const long long e0 = a.off[v], e1 = a.off[v + 1];
        bool ready = true;
        for (long long e = e0; e < e1 && ready; ++e) {
            const int u = a.col[e];
            if (u != v && colour_priority((unsigned long long)(u - vo)) > pv && colour[u] < 0) ready = false;
        }
        if (!ready) {
            ++left;
            continue;
        }
        // least colour not held by a higher-priority neighbour, 64 at a time
        for (int base = 0;; base += 64) {
            unsigned long long used = 0;
            for (long long e = e0; e < e1; ++e) {
                const int u = a.col[e];
                if (u == v || colour_priority((unsigned long long)(u - vo)) <= pv) continue;
                const int cu = colour[u] - base;
                if (cu >= 0 && cu < 64) used |= 1ull << cu;
            }
            if (~used) {
                a.colour[v] = base + __ffsll((long long)~used) - 1;
                break;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) left += __shfl_xor_sync(0xffffffffu, left, o);
    if ((threadIdx.x & 31) == 0 && left) atomicAdd(a.flag, left);
}

__global__ void k_colour_max(ColourArgs a)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    int m = -1;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += stride) m = max(m, a.colour[v]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(a.flag, m + 1);
}

// Per class: vertices (cnt[c]) and CSR entries (cnt[classes + 1 + c]).
__global__ void k_colour_count(ColourArgs a, int classes)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += stride) {
        const int c = a.colour[v];
        atomicAdd(reinterpret_cast<unsigned long long*>(a.cnt + c), 1ull);
        atomicAdd(reinterpret_cast<unsigned long long*>(a.cnt + classes + 1 + c),
                  (unsigned long long)(a.off[v + 1] - a.off[v]));
    }
}

// Lists the vertices and the CSR entries of each class (cnt now holds the
// running positions; the order inside a class does not matter).
__global__ void k_colour_place(ColourArgs a, int classes)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += stride) {
        const int c = a.colour[v];
        const long long d = a.off[v + 1] - a.off[v];
        const long long p = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(a.cnt + c), 1ull);
        a.vlist[p] = (int)v;
        const long long q = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(a.cnt + classes + 1 + c),
                                                 (unsigned long long)d);
        for (long long t = 0; t < d; ++t) a.eidx[q + t] = (int)(a.off[v] + t);
    }
}

}  // namespace

cudaError_t launch_colouring(const ColourArgs& a, int* classes, cudaStream_t s)
{
    const int g = grid_for(a.n);
    k_colour_init<<<g, kSetupBlock, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    // rounds until every vertex is coloured; each round colours at least the
    // uncoloured vertex of highest priority, so n rounds always suffice
    for (long long round = 0; e == cudaSuccess; ++round) {
        if (round > a.n) return cudaErrorUnknown;
        e = cudaMemsetAsync(a.flag, 0, sizeof(int), s);
        if (e != cudaSuccess) return e;
        k_colour_round<<<g, kSetupBlock, 0, s>>>(a);
        int left = 0;
        e = cudaMemcpyAsync(&left, a.flag, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        if (left == 0) break;
    }
    e = cudaMemsetAsync(a.flag, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_colour_max<<<g, kSetupBlock, 0, s>>>(a);
    int nc = 0;
    e = cudaMemcpyAsync(&nc, a.flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (nc < 1) nc = 1;
    e = cudaMemsetAsync(a.cnt, 0, sizeof(long long) * 2 * ((size_t)nc + 1), s);
    if (e != cudaSuccess) return e;
    k_colour_count<<<g, kSetupBlock, 0, s>>>(a, nc);
    std::vector<long long> cnt(2 * ((size_t)nc + 1));
    e = cudaMemcpyAsync(cnt.data(), a.cnt, sizeof(long long) * cnt.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    // class offsets: exclusive prefix sums of the counts
    std::vector<int> voff((size_t)nc + 1, 0);
    std::vector<long long> eoff((size_t)nc + 1, 0), pos(2 * ((size_t)nc + 1), 0);
    for (int c = 0; c < nc; ++c) {
        voff[c + 1] = voff[c] + (int)cnt[c];
        eoff[c + 1] = eoff[c] + cnt[nc + 1 + c];
        pos[c] = voff[c];
        pos[nc + 1 + c] = eoff[c];
    }
    e = cudaMemcpyAsync(a.voff, voff.data(), sizeof(int) * voff.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(a.eoff, eoff.data(), sizeof(long long) * eoff.size(),
                                              cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(a.cnt, pos.data(), sizeof(long long) * pos.size(),
                                              cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    k_colour_place<<<g, kSetupBlock, 0, s>>>(a, nc);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // pos, voff, eoff are host vectors
    *classes = nc;
    return e;
}

cudaError_t launch_assemble(const AssemblyArgs& a, cudaStream_t s)
{
    k_fill_jid<<<grid_for(a.n), kSetupBlock, 0, s>>>(a);
    k_assemble_off<<<grid_for(a.n), kSetupBlock, 0, s>>>(a);
    return cudaGetLastError();
}

// Second half of the assembly, run once the offsets are known to be valid.
cudaError_t launch_assemble_edges(const AssemblyArgs& a, cudaStream_t s)
{
    k_fill_src<<<grid_for(a.n), kSetupBlock, 0, s>>>(a);
    k_assemble_col<<<grid_for(a.nnz), kSetupBlock, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_compact_labels(const LabelArgs& a, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(a.G, 0xff, sizeof(int) * (size_t)a.rows, s);
    if (e != cudaSuccess) return e;
    return launch_label_kernels(a, s);
}

cudaError_t launch_label_kernels(const LabelArgs& a, cudaStream_t s)
{
    LSlot* m = static_cast<LSlot*>(a.lmap);
    const unsigned long long cap = a.lmask + 1;
    k_lmap_clear<<<grid_for((long long)cap), kSetupBlock, 0, s>>>(m, cap);
    k_label_insert<<<grid_for(a.total), kSetupBlock, 0, s>>>(a);
    k_label_assign<<<grid_for(a.total), kSetupBlock, 0, s>>>(a);
    k_label_sumsq<<<grid_for((long long)cap), kSetupBlock, smem_jobs_bytes(a.jobs), s>>>(a, cap);
    return cudaGetLastError();
}

cudaError_t launch_init_state(const SweepArgs& a, cudaStream_t s)
{
    k_init_state<<<grid_for(a.n), kSetupBlock, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_singleton_summaries(const SweepArgs& a, long long rows, cudaStream_t s)
{
    k_summ_singletons<<<grid_for(rows), kSetupBlock, 0, s>>>(a, rows);
    return cudaGetLastError();
}

cudaError_t launch_state_from_ids(const SweepArgs& a, cudaStream_t s)
{
    k_sizes_zero<<<grid_for(a.n), kSetupBlock, 0, s>>>(a);
    k_count_sizes<<<grid_for(a.n), kSetupBlock, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_table_rebuild(const SweepArgs& a, long long rows, bool conditional, cudaStream_t s, bool eval)
{
    const int c = conditional ? 1 : 0;
    const int nb = (int)((a.n + 1023) / 1024);
    k_table_clear<<<grid_for(std::max((long long)a.mask_max + 1, rows)), kSetupBlock, 0, s>>>(a, rows, c);
    k_scan_blocks<<<nb, 1024, 0, s>>>(a, c);
    k_scan_sums<<<1, 1024, 0, s>>>(a, nb, c);
    k_scan_write<<<nb, 1024, 0, s>>>(a, c);
    k_members_scatter<<<grid_for(a.n), kSetupBlock, 0, s>>>(a, c);
    k_table_build<<<grid_for(a.n), kSetupBlock, eval ? smem_jobs_bytes(a.jobs) : 0, s>>>(a, c, eval ? 1 : 0);
    k_build_check<<<1, 256, 0, s>>>(a, c);
    k_summ_top<<<grid_for((long long)a.mask_max + 1), kSetupBlock, eval ? smem_jobs_bytes(a.jobs) : 0, s>>>(a, c,
                                                                                                 eval ? 1 : 0);
    k_table_done<<<1, 1, 0, s>>>(a.st, c);
    return cudaGetLastError();
}

cudaError_t launch_objective_recompute(const SweepArgs& a, cudaStream_t s)
{
    k_zero_recompute<<<grid_for(a.jobs), kSetupBlock, 0, s>>>(a);
    const long long work = (long long)a.mask_max + 1 > a.n ? (long long)a.mask_max + 1 : a.n;
    k_objective_recompute<<<grid_for(work), kSetupBlock, smem_jobs_bytes(a.jobs), s>>>(a);
    return cudaGetLastError();
}

}  // namespace ccg
