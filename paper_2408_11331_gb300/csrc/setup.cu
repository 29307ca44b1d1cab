// Setup of one consensus job (The algorithm: Initialization) and the table
// maintenance kernels: input validation, per-partition label compaction into
// the vertex-major membership matrix, the singleton state, the contingency
// hash build, and the from-scratch objective used for checks.
#include <climits>

#include "cc_internal.cuh"

namespace ccg {

namespace {

constexpr int kSetupBlock = 256;

inline int grid_for(long long work, int per_block = kSetupBlock, int max_blocks = 152 * 16)
{
    long long b = (work + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

// (partition, raw label) -> least vertex carrying it, and the class size.
struct __align__(16) LSlot {
    unsigned long long key;
    int rep;
    int cnt;
};

__device__ __forceinline__ long long warp_sum64(long long x)
{
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Block-wide sum of x, added to *out by one thread.  Every thread of the block calls it.
__device__ void block_add64(long long x, long long* out)
{
    __shared__ long long part[32];
    x = warp_sum64(x);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) part[w] = x;
    __syncthreads();
    if (w == 0) {
        long long y = lane < (int)(blockDim.x >> 5) ? part[lane] : 0;
        y = warp_sum64(y);
        if (lane == 0 && y != 0) atomicAdd(reinterpret_cast<unsigned long long*>(out), (unsigned long long)y);
    }
    __syncthreads();
}

__global__ void k_validate(int n, long long nnz, const long long* __restrict__ off,
                           const int* __restrict__ col, DevState* st)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long v = t0; v <= n; v += stride) {
        long long o = off[v];
        bool bad = (v == 0 && o != 0) || (v == n && o != nnz) || (v < n && off[v + 1] < o);
        if (bad) set_err(st, CC_ERR_INVALID);
    }
    for (long long e = t0; e < nnz; e += stride) {
        int u = col[e];
        if (u < 0 || u >= n) set_err(st, CC_ERR_INVALID);
    }
}

__global__ void k_fill_src(int n, const long long* __restrict__ off, int* src)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        for (long long e = off[v]; e < off[v + 1]; ++e) src[e] = (int)v;
}

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

// labels is partition-major: entry t = i*n + v.
__global__ void k_label_insert(int n, int k, const int* __restrict__ labels, LSlot* m, unsigned long long mask,
                               DevState* st)
{
    const long long total = (long long)n * k;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const int i = (int)(t / n), v = (int)(t - (long long)i * n);
        const unsigned long long key = ((unsigned long long)(unsigned)i << 32) | (unsigned)labels[t];
        long long s = lmap_slot(m, mask, key, true);
        if (s < 0) { set_err(st, CC_ERR_TABLE_FULL); continue; }
        atomicMin(&m[s].rep, v);
        atomicAdd(&m[s].cnt, 1);
    }
}

// G[v][i] = (i << lshift) | rep(i, label).  Tiles of 32 vertices x up to 32 partitions are
// transposed through shared memory so both the label reads and the row writes
// are coalesced.
__global__ void k_label_assign(int n, int k, int kp, int lshift, const int* __restrict__ labels, const LSlot* m,
                               unsigned long long mask, int* __restrict__ G, DevState* st)
{
    __shared__ int tile[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    const long long vt = ((long long)n + 31) / 32, it = ((long long)kp + 31) / 32;
    for (long long b = blockIdx.x; b < vt * it; b += gridDim.x) {
        const long long v0 = (b / it) * 32;
        const int i0 = (int)(b % it) * 32;
        for (int r = ty; r < 32; r += 8) {
            const int i = i0 + r;
            const long long v = v0 + tx;
            int g = -1;
            if (i < k && v < n) {
                const unsigned long long key = ((unsigned long long)(unsigned)i << 32) | (unsigned)labels[(long long)i * n + v];
                long long s = lmap_slot(const_cast<LSlot*>(m), mask, key, false);
                if (s < 0) set_err(st, CC_ERR_INVALID);
                else g = (i << lshift) | m[s].rep;
            }
            tile[r][tx] = g;
        }
        __syncthreads();
        for (int r = ty; r < 32; r += 8) {
            const long long v = v0 + r;
            const int i = i0 + tx;
            if (v < n && i < kp) G[v * kp + i] = tile[tx][r];
        }
        __syncthreads();
    }
}

__global__ void k_label_sumsq(const LSlot* m, unsigned long long cap, DevState* st)
{
    long long acc = 0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; s < cap; s += stride) {
        long long c = m[s].cnt;
        acc += c * c;
    }
    block_add64(acc, &st->partition_sq);
}

__global__ void k_init_state(int n, int* C, int* size, int* dsize, unsigned long long* best)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        C[v] = (int)v;
        size[v] = 1;
        dsize[v] = 0;
        best[v] = kEmpty;
    }
}

// Sizes from a given consensus; ids outside [0, n) set an error.
__global__ void k_sizes_from_ids(int n, const int* __restrict__ C, int* size, int* dsize,
                                 unsigned long long* best, DevState* st)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        size[v] = 0;
        dsize[v] = 0;
        best[v] = kEmpty;
    }
}

__global__ void k_count_sizes(int n, const int* __restrict__ C, int* size, DevState* st)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int c = C[v];
        if (c < 0 || c >= n) set_err(st, CC_ERR_INVALID);
        else atomicAdd(&size[c], 1);
    }
}

// ---- table rebuild ------------------------------------------------------
// The table is rebuilt from C alone: clear the capacity being built, list the
// vertices cluster by cluster (counting sort: an exclusive scan of the sizes
// gives each cluster's first position), then insert the keys with partitions
// innermost per member, so that the 32 lanes of a warp hold consecutive
// members of (mostly) one cluster for one partition: equal keys are merged
// with __match_any_sync and added with one atomic.  All kernels are skipped
// unless a rebuild is pending (conditional) and run unconditionally at reset.

__device__ __forceinline__ bool rebuild_off(const DevState* st, int conditional)
{
    return conditional && (!st->rebuild || st->err);
}

// Clears the slots of the capacity being built (st->new_mask + 1 of them), and
// the staged size deltas after an abandoned sweep.
__global__ void k_table_clear(Slot* t, int* dsize, int n, const DevState* st, int conditional)
{
    if (rebuild_off(st, conditional)) return;
    const unsigned long long cap = st->new_mask + 1;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long t0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (unsigned long long s = t0; s < cap; s += stride)
        reinterpret_cast<ulonglong2*>(t)[s] = make_ulonglong2(kEmpty, 0ull);
    if (st->abort)
        for (unsigned long long v = t0; v < (unsigned long long)n; v += stride) dsize[v] = 0;
}

__global__ void k_table_reset_counters(DevState* st, int conditional)
{
    if (rebuild_off(st, conditional)) return;
    st->used = 0;
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
__global__ void __launch_bounds__(1024) k_scan_blocks(const int* __restrict__ in, int n, int* bsum,
                                                      const DevState* st, int conditional)
{
    if (rebuild_off(st, conditional)) return;
    __shared__ int wsum[32];
    const int i = blockIdx.x * 1024 + threadIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = i < n ? in[i] : 0;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int y = wsum[lane];
        for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
        if (lane == 0) bsum[blockIdx.x] = y;
    }
}

// Exclusive scan of the nb block sums in place (one block, 1024 threads, each
// owning a contiguous run).
__global__ void __launch_bounds__(1024) k_scan_sums(int nb, int* bsum, const DevState* st, int conditional)
{
    if (rebuild_off(st, conditional)) return;
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int per = (nb + 1023) / 1024;
    const int lo = threadIdx.x * per, hi = min(nb, lo + per);
    int sum = 0;
    for (int b = lo; b < hi; ++b) sum += bsum[b];
    int x = warp_incl_scan(sum, lane);
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) wsum[lane] = warp_incl_scan(wsum[lane], lane);
    __syncthreads();
    int run = x - sum + (w > 0 ? wsum[w - 1] : 0);
    for (int b = lo; b < hi; ++b) {
        const int y = bsum[b];
        bsum[b] = run;
        run += y;
    }
}

// cursor[c] = exclusive prefix of size[] (the first position of cluster c).
__global__ void __launch_bounds__(1024) k_scan_write(const int* __restrict__ in, int n, const int* __restrict__ bsum,
                                                     int* out, const DevState* st, int conditional)
{
    if (rebuild_off(st, conditional)) return;
    __shared__ int wsum[32];
    const int i = blockIdx.x * 1024 + threadIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int v = i < n ? in[i] : 0;
    int x = warp_incl_scan(v, lane);
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) wsum[lane] = warp_incl_scan(wsum[lane], lane);
    __syncthreads();
    if (i < n) out[i] = bsum[blockIdx.x] + x - v + (w > 0 ? wsum[w - 1] : 0);
}

__global__ void k_members_scatter(int n, const int* __restrict__ C, int* cursor, int* members, const DevState* st,
                                  int conditional)
{
    if (rebuild_off(st, conditional)) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int pos = atomicAdd(&cursor[C[v]], 1);
        if (pos < n) members[pos] = (int)v;
        else set_err(const_cast<DevState*>(st), CC_ERR_INVALID);  // sizes inconsistent with C
    }
}

__global__ void k_table_build(SweepArgs a, int conditional)
{
    DevState* st = a.st;
    if (rebuild_off(st, conditional)) return;
    const unsigned long long mask = st->new_mask;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < a.n; base += stride) {
        const long long m = base + threadIdx.x;
        const bool valid = m < a.n;
        int v = 0, c = 0;
        if (valid) {
            v = a.members[m];
            c = a.C[v];
        }
        const int* row = a.G + (long long)v * a.kp;
        for (int i = 0; i < a.k; ++i) {
            const unsigned long long key = valid ? ckey(c, row[i]) : kEmpty;
            const unsigned same = __match_any_sync(0xffffffffu, key);
            bool ins = false;
            if (valid && (__ffs(same) - 1) == lane) {
                const long long s = table_find_or_insert(a.table, mask, key, &ins);
                if (s < 0) set_err(st, CC_ERR_TABLE_FULL);
                else atomicAdd(&a.table[s].cnt, __popc(same));
            }
            const unsigned mi = __ballot_sync(0xffffffffu, ins);
            if (lane == 0 && mi) atomicAdd(&st->used, (unsigned long long)__popc(mi));
        }
    }
}

// Summary rows of the rebuilt table.  The first 8 bytes of a row are read as
// one unsigned 64-bit value (count << 32 | label id), so an atomic maximum
// over the slots of a (cluster, partition) leaves the most frequent label and
// its count (ties to the larger id); a second pass takes the largest count of
// the other labels.
__global__ void k_summ_clear(int4* summ, long long rows, const DevState* st, int conditional)
{
    if (rebuild_off(st, conditional)) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += stride)
        summ[r] = make_int4(0, 0, 0, 0);
}

// In the first rebuild of a heavy sweep this pass also adds -2 sum n^2 over
// the new keys to st->recompute (the table part of F').
__global__ void k_summ_top(SweepArgs a, int conditional)
{
    DevState* st = a.st;
    if (rebuild_off(st, conditional)) return;
    const bool eval = st->heavy && !st->rollback;
    const unsigned long long cap = st->new_mask + 1;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    long long sq = 0;
    for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; s < cap; s += stride) {
        const ulonglong2 e = reinterpret_cast<const ulonglong2*>(a.table)[s];
        const int cnt = (int)(unsigned)(e.y & 0xffffffffull);
        if (e.x == kEmpty || cnt <= 0) continue;
        const int x = (int)(e.x >> 32), g = (int)(unsigned)(e.x & 0xffffffffull);
        const long long row = (long long)x * a.kp + (g >> a.lshift);
        atomicMax(reinterpret_cast<unsigned long long*>(a.summ + row), ((unsigned long long)(unsigned)cnt << 32) | (unsigned)g);
        sq += (long long)cnt * cnt;
    }
    if (eval) block_add64(-2 * sq, &st->recompute);
}

__global__ void k_summ_second(SweepArgs a, int conditional)
{
    const DevState* st = a.st;
    if (rebuild_off(st, conditional)) return;
    const unsigned long long cap = st->new_mask + 1;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; s < cap; s += stride) {
        const ulonglong2 e = reinterpret_cast<const ulonglong2*>(a.table)[s];
        const int cnt = (int)(unsigned)(e.y & 0xffffffffull);
        if (e.x == kEmpty || cnt <= 0) continue;
        const int x = (int)(e.x >> 32), g = (int)(unsigned)(e.x & 0xffffffffull);
        int4* S = a.summ + (long long)x * a.kp + (g >> a.lshift);
        if (S->x != g) atomicMax(&S->z, cnt);
    }
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

__global__ void k_objective_recompute(SweepArgs a)
{
    long long acc = 0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long t0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (unsigned long long v = t0; v < (unsigned long long)a.n; v += stride) {
        long long s = a.size[v];
        acc += (long long)a.k * s * s;
    }
    const unsigned long long mask = a.st->mask;
    for (unsigned long long s = t0; s <= mask; s += stride) {
        if (a.table[s].key != kEmpty) {
            long long c = a.table[s].cnt;
            acc -= 2 * c * c;
        }
    }
    block_add64(acc, &a.st->recompute);
}

}  // namespace

cudaError_t launch_validate(int n, long long nnz, const long long* off, const int* col, DevState* st, cudaStream_t s)
{
    k_validate<<<grid_for(nnz > n ? nnz : (long long)n + 1), kSetupBlock, 0, s>>>(n, nnz, off, col, st);
    return cudaGetLastError();
}

cudaError_t launch_fill_src(int n, const long long* off, int* src, cudaStream_t s)
{
    k_fill_src<<<grid_for(n), kSetupBlock, 0, s>>>(n, off, src);
    return cudaGetLastError();
}

// lmap: 16-byte slots, lmask + 1 of them (caller-owned scratch, >= 2 k n).
cudaError_t launch_compact_labels(int n, int k, int kp, int lshift, const int* labels, int* G, void* lmap,
                                  unsigned long long lmask, DevState* st, cudaStream_t s)
{
    LSlot* m = static_cast<LSlot*>(lmap);
    const unsigned long long cap = lmask + 1;
    k_lmap_clear<<<grid_for((long long)cap), kSetupBlock, 0, s>>>(m, cap);
    k_label_insert<<<grid_for((long long)n * k), kSetupBlock, 0, s>>>(n, k, labels, m, lmask, st);
    const long long tiles = ((long long)n + 31) / 32 * (((long long)kp + 31) / 32);
    k_label_assign<<<(int)(tiles < 152 * 16 ? tiles : 152 * 16), 256, 0, s>>>(n, k, kp, lshift, labels, m, lmask, G, st);
    k_label_sumsq<<<grid_for((long long)cap), kSetupBlock, 0, s>>>(m, cap, st);
    return cudaGetLastError();
}

__global__ void k_summ_singletons(SweepArgs a)
{
    const long long rows = (long long)a.n * a.kp;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += stride) {
        const int i = (int)(r % a.kp);
        a.summ[r] = i < a.k ? make_int4(a.G[r], 1, 0, 0) : make_int4(-1, 0, 0, 0);
    }
}

cudaError_t launch_singleton_summaries(const SweepArgs& a, cudaStream_t s)
{
    k_summ_singletons<<<grid_for((long long)a.n * a.kp), kSetupBlock, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_init_state(const SweepArgs& a, cudaStream_t s)
{
    k_init_state<<<grid_for(a.n), kSetupBlock, 0, s>>>(a.n, a.C, a.size, a.dsize, a.best);
    return cudaGetLastError();
}

cudaError_t launch_state_from_ids(const SweepArgs& a, cudaStream_t s)
{
    k_sizes_from_ids<<<grid_for(a.n), kSetupBlock, 0, s>>>(a.n, a.C, a.size, a.dsize, a.best, a.st);
    k_count_sizes<<<grid_for(a.n), kSetupBlock, 0, s>>>(a.n, a.C, a.size, a.st);
    return cudaGetLastError();
}

cudaError_t launch_table_rebuild(const SweepArgs& a, bool conditional, cudaStream_t s)
{
    const int c = conditional ? 1 : 0;
    const int nb = (a.n + 1023) / 1024;
    k_table_clear<<<grid_for((long long)a.mask_max + 1), kSetupBlock, 0, s>>>(a.table, a.dsize, a.n, a.st, c);
    k_table_reset_counters<<<1, 1, 0, s>>>(a.st, c);
    k_scan_blocks<<<nb, 1024, 0, s>>>(a.size, a.n, a.bsum, a.st, c);
    k_scan_sums<<<1, 1024, 0, s>>>(nb, a.bsum, a.st, c);
    k_scan_write<<<nb, 1024, 0, s>>>(a.size, a.n, a.bsum, a.cursor, a.st, c);
    k_members_scatter<<<grid_for(a.n), kSetupBlock, 0, s>>>(a.n, a.C, a.cursor, a.members, a.st, c);
    k_table_build<<<grid_for(a.n), kSetupBlock, 0, s>>>(a, c);
    k_summ_clear<<<grid_for((long long)a.n * a.kp), kSetupBlock, 0, s>>>(a.summ, (long long)a.n * a.kp, a.st, c);
    k_summ_top<<<grid_for((long long)a.mask_max + 1), kSetupBlock, 0, s>>>(a, c);
    k_summ_second<<<grid_for((long long)a.mask_max + 1), kSetupBlock, 0, s>>>(a, c);
    k_table_done<<<1, 1, 0, s>>>(a.st, c);
    return cudaGetLastError();
}

cudaError_t launch_objective_recompute(const SweepArgs& a, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(&a.st->recompute, 0, sizeof(long long), s);
    if (e != cudaSuccess) return e;
    long long work = (long long)a.mask_max + 1 > a.n ? (long long)a.mask_max + 1 : a.n;
    k_objective_recompute<<<grid_for(work), kSetupBlock, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace ccg
