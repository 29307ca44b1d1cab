// Setup of the jobs of a context (The algorithm: Initialization) and the
// table maintenance kernels: union assembly with input validation, per-job
// label compaction into the vertex-major membership matrix, the singleton
// state, the contingency hash rebuild with its summary rows, and the
// from-scratch objective used for checks.
#include <algorithm>
#include <atomic>
#include <climits>

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
        a.summ[r] = g >= 0 ? make_int2(g, 1) : make_int2(-1, 0);
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
// after an abandoned sweep.
__global__ void k_table_clear(SweepArgs a, long long rows, int conditional)
{
    DevState* st = a.st;
    if (rebuild_off(st, conditional)) return;
    const unsigned long long cap = st->new_mask + 1;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long t0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (unsigned long long s = t0; s < cap; s += stride)
        reinterpret_cast<ulonglong2*>(a.table)[s] = make_ulonglong2(kEmpty, 0ull);
    for (unsigned long long r = t0; r < (unsigned long long)rows; r += stride) a.summ[r] = make_int2(0, 0);
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

__global__ void k_table_build(SweepArgs a, int conditional)
{
    DevState* st = a.st;
    if (rebuild_off(st, conditional)) return;
    __shared__ unsigned long long s_used;
    if (threadIdx.x == 0) s_used = 0;
    __syncthreads();
    const unsigned long long mask = st->new_mask;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    unsigned long long used = 0;  // slots this warp created (lane 0 counts)
    for (long long base = (long long)blockIdx.x * blockDim.x; base < a.n; base += stride) {
        const long long m = base + threadIdx.x;
        const bool valid = m < a.n;
        int v = 0, c = 0, k = 0;
        const int* row = a.G;
        if (valid) {
            v = a.members[m];
            c = a.C[v];
            const JobInfo& J = a.job[a.jid[v]];
            k = J.k;
            row = a.G + row_of(J, v);
        }
        for (int i = 0; i < a.kmax; ++i) {
            const bool on = valid && i < k;
            const unsigned long long key = on ? ckey(c, row[i]) : kEmpty;
            const unsigned same = __match_any_sync(0xffffffffu, key);
            bool ins = false;
            if (on && (__ffs(same) - 1) == lane) {
                if (table_build_add(a.table, mask, key, __popc(same), &ins) < 0) set_err(st, CC_ERR_TABLE_FULL);
            }
            used += __popc(__ballot_sync(0xffffffffu, ins));
        }
    }
    // one add per block: st->used is a single word that every block updates
    if (lane == 0 && used) atomicAdd(&s_used, used);
    __syncthreads();
    if (threadIdx.x == 0 && s_used) atomicAdd(&st->used, s_used);
}

// Summary rows of the rebuilt table.  A row entry is read as one unsigned
// 64-bit value (count << 32 | label id), so an atomic maximum over the slots
// of a (cluster, partition) leaves the most frequent label and its count
// (ties to the larger id).
// With eval set (the first rebuild of a heavy sweep) this pass also adds
// -2 sum n^2 over the new keys to each job's recompute (the table part of F').
__global__ void k_summ_top(SweepArgs a, int conditional, int eval)
{
    extern __shared__ long long dyn_jobs[];
    DevState* st = a.st;
    if (rebuild_off(st, conditional)) return;
    const bool ev = eval && st->heavy;
    JobAcc acc(ev ? job_smem_init(a.jobs, dyn_jobs) : nullptr, &a.js[0].recompute, kJobStride);
    const unsigned long long cap = st->new_mask + 1;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; s < cap; s += stride) {
        const ulonglong2 e = reinterpret_cast<const ulonglong2*>(a.table)[s];
        const int cnt = (int)(unsigned)(e.y & 0xffffffffull);
        if (e.x == kEmpty || cnt <= 0) continue;
        const int x = (int)(e.x >> 32), g = (int)(unsigned)(e.x & 0xffffffffull);
        const int job = a.jid[x];
        const JobInfo& J = a.job[job];
        atomicMax(reinterpret_cast<unsigned long long*>(a.summ + row_of(J, x) + (g >> J.lshift)),
                  ((unsigned long long)(unsigned)cnt << 32) | (unsigned)g);
        if (ev) acc.add(job, -2LL * cnt * cnt);
    }
    if (ev) job_acc_finish(acc, a.jobs);
}

__global__ void k_table_done(DevState* st, int conditional)
{
    if (rebuild_off(st, conditional)) return;
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

}  // namespace

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
    LSlot* m = static_cast<LSlot*>(a.lmap);
    const unsigned long long cap = a.lmask + 1;
    cudaError_t e = cudaMemsetAsync(a.G, 0xff, sizeof(int) * (size_t)a.rows, s);
    if (e != cudaSuccess) return e;
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
    k_table_build<<<grid_for(a.n), kSetupBlock, 0, s>>>(a, c);
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
