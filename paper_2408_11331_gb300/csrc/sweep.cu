// One synchronous local-move sweep (Methods, "Parallel algorithm"), as a fixed
// sequence of kernels on one stream so that it can be captured in a CUDA graph:
//
//   begin       per-sweep counters; the sweep is skipped once the run has stopped
//   own/edges/  best move of every vertex against the sweep-start state
//   collect     (Eq. objective4 with the gain of Eq. objective3): A_a per
//               vertex, then one lane group per CSR entry bidding its move,
//               then the proposal list
//   stage       singleton guard; stage the size and count deltas of the kept
//               proposals P1 in the table (inserting target keys)
//   eval        exact dF of applying P1 at once, from the staged deltas
//   decide      commit P1 if dF < 0, else fall back to the matching of P
//   commit      fold the staged deltas in (P1), or clear them and bid for the
//               matching (fallback)
//   match_*     commit the proposals that hold the least (dD, v) at both ends
//   end         objective, history record, stop and rebuild decisions
//   rebuild     (conditional) rebuild the contingency hash without dead keys
//
// Gain of v moving from its cluster a to b (Eq. objective3, u = v excluded):
//   dD = 2 (A_a - k - A_b) - k (|a| - 1 - |b|),   A_x = sum_i n(x, i, l_i(v)),
// and the move changes F by 2 dD.  For a singleton candidate {u}, A_x is the
// number of partitions in which u and v agree, read from u's label row; other
// candidates take k probes of the contingency hash.
#include "cc_internal.cuh"

namespace ccg {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// (dD, id) packed so that unsigned order is (dD, id) order: dD with its sign
// bit flipped in the high word.
__device__ __forceinline__ unsigned long long pack_key(int dD, int id)
{
    return ((unsigned long long)((unsigned)dD ^ 0x80000000u) << 32) | (unsigned)id;
}

__device__ __forceinline__ int key_gain(unsigned long long key)
{
    return (int)((unsigned)(key >> 32) ^ 0x80000000u);
}

__device__ __forceinline__ long long warp_sum64(long long x)
{
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

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

// Count under key given the slot h = hash(key) & mask already loaded as e.
__device__ __forceinline__ int resolve(const Slot* t, unsigned long long mask, unsigned long long key,
                                       unsigned long long h, ulonglong2 e)
{
    for (unsigned long long p = 0; p <= mask; ++p) {
        if (e.x == key) return (int)(unsigned)(e.y & 0xffffffffull);
        if (e.x == kEmpty) return 0;
        h = (h + 1) & mask;
        e = __ldg(reinterpret_cast<const ulonglong2*>(t + h));
    }
    return 0;
}

__global__ void k_run_begin(DevState* st, int limit)
{
    st->stop = 0;
    st->run_sweeps = 0;
    st->run_limit = limit;
}

__global__ void k_begin(DevState* st)
{
    st->skip = (st->stop || st->err) ? 1 : 0;
    st->overflow = 0;
    st->nprop = 0;
    st->np1 = 0;
    st->dF = 0;
    st->dF_p1 = 0;
    st->moves = 0;
    st->tile_ctr = 0;
    st->mode = 0;
}

constexpr int kInflight = 4;  // loads per lane issued before the first is used

__device__ __forceinline__ int group_sum(int x, int gs)
{
    for (int o = gs >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

// Summary part of A_x(v) for a non-singleton cluster x, lanes of a group over
// the partitions i = l, l + gs, ...: ex = sum of m where v carries the row's
// label d (exact there), ub = ex + sum of m2 elsewhere (an upper bound on
// A_x), nq = number of partitions where v does not carry d.
__device__ __forceinline__ void summary_part(const SweepArgs& a, const int* __restrict__ gv, int x, int l, int gs,
                                             int& ex, int& ub, int& nq)
{
    ex = 0;
    ub = 0;
    nq = 0;
    const int4* S = a.summ + (long long)x * a.kp;
    for (int i0 = l; i0 < a.k; i0 += gs * kInflight) {
        int4 r[kInflight];
        int g[kInflight];
#pragma unroll
        for (int b = 0; b < kInflight; ++b) {
            const int i = i0 + b * gs;
            r[b] = make_int4(-1, 0, 0, 0);
            g[b] = -2;
            if (i < a.k) {
                r[b] = __ldg(S + i);
                g[b] = __ldg(gv + i);
            }
        }
#pragma unroll
        for (int b = 0; b < kInflight; ++b) {
            if (i0 + b * gs < a.k) {
                const bool eq = g[b] == r[b].x;
                ex += eq ? r[b].y : 0;
                ub += eq ? r[b].y : r[b].z;
                nq += eq ? 0 : 1;
            }
        }
    }
}

// Exact counts of the partitions the summary leaves open (v does not carry
// the row's label and another label may be present), by hash probes.
__device__ __forceinline__ int probe_part(const SweepArgs& a, const Slot* __restrict__ table, unsigned long long mask,
                                          const int* __restrict__ gv, int x, int l, int gs)
{
    const int4* S = a.summ + (long long)x * a.kp;
    int acc = 0;
    for (int i0 = l; i0 < a.k; i0 += gs * kInflight) {
        unsigned long long key[kInflight], h[kInflight];
        ulonglong2 ev[kInflight];
        bool on[kInflight];
#pragma unroll
        for (int b = 0; b < kInflight; ++b) {
            const int i = i0 + b * gs;
            on[b] = false;
            key[b] = 0;
            h[b] = 0;
            ev[b] = make_ulonglong2(kEmpty, 0ull);
            if (i < a.k) {
                const int4 r = __ldg(S + i);
                const int g = __ldg(gv + i);
                on[b] = g != r.x && r.z > 0;
                if (on[b]) {
                    key[b] = ckey(x, g);
                    h[b] = hash_key(key[b]) & mask;
                    ev[b] = __ldg(reinterpret_cast<const ulonglong2*>(table + h[b]));
                }
            }
        }
#pragma unroll
        for (int b = 0; b < kInflight; ++b)
            if (on[b]) acc += resolve(table, mask, key[b], h[b], ev[b]);
    }
    return acc;
}

// Partitions in which u and v carry the same label, plus the padding entries
// of this lane's quads: the two label rows compared as int4 quads.
__device__ __forceinline__ int row_part(const SweepArgs& a, int u, int v, int l, int gs)
{
    const int4* gu = reinterpret_cast<const int4*>(a.G + (long long)u * a.kp);
    const int4* gw = reinterpret_cast<const int4*>(a.G + (long long)v * a.kp);
    const int kq = a.kp >> 2;
    int acc = 0;
    for (int q0 = l; q0 < kq; q0 += gs * kInflight) {
        int4 r[kInflight], s[kInflight];
#pragma unroll
        for (int b = 0; b < kInflight; ++b) {
            const int q = q0 + b * gs;
            r[b] = make_int4(-1, -1, -1, -1);
            s[b] = make_int4(-3, -3, -3, -3);
            if (q < kq) {
                r[b] = __ldg(gu + q);
                s[b] = __ldg(gw + q);
            }
        }
#pragma unroll
        for (int b = 0; b < kInflight; ++b)
            acc += (r[b].x == s[b].x) + (r[b].y == s[b].y) + (r[b].z == s[b].z) + (r[b].w == s[b].w);
    }
    return acc;  // includes the kp - k padding entries (-1 in every row)
}

// Lanes per vertex (k_own) or per edge (k_edges): about five partitions per lane.
__host__ __device__ __forceinline__ int lanes_per_item(int k)
{
    int gs = 1;
    while (gs < 32 && gs * 5 < k) gs <<= 1;
    return gs;
}

// A_a for every vertex: k for a singleton, else the summary part of its own
// cluster plus probes of the open partitions.  One group of lanes per vertex.
__global__ void __launch_bounds__(kBlock) k_own(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip) return;
    const unsigned long long mask = st->mask;
    const int gs = lanes_per_item(a.k);
    const int lane = threadIdx.x & 31, l = lane & (gs - 1);
    const long long groups = (long long)gridDim.x * blockDim.x / gs;
    for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x - lane) / gs; base < a.n;
         base += groups) {
        const long long v = base + lane / gs;
        const bool valid = v < a.n;
        const int cv = valid ? __ldg(a.C + v) : 0;
        const int sa = valid ? __ldg(a.size + cv) : 1;
        const int* gv = a.G + (valid ? v : 0) * (long long)a.kp;
        int ex = 0, ub = 0, nq = 0, pb = 0;
        if (sa > 1) {
            summary_part(a, gv, cv, l, gs, ex, ub, nq);
            pb = probe_part(a, a.table, mask, gv, cv, l, gs);
        }
        const int A = group_sum(ex + pb, gs);
        if (valid && l == 0) a.aown[v] = sa > 1 ? A : a.k;
    }
}

// Foreign CSR entries of one warp, compacted in shared memory.
struct EdgeScratch {
    int v[32], u[32], x[32], sx[32], sa[32], Aa[32];
};

// CSR entries 32 at a time per warp: each lane reads one entry (v, u) and
// keeps it if u lies in another cluster than v (self-loops and repeats of the
// same (v, C[u]) inside the warp are dropped); the kept entries are then
// scored by groups of lanes.  A singleton {u} is scored from the two label
// rows; another cluster from its summary rows, then (unless the lower bound on
// dD from the summary is already >= 0) from probes of the open partitions.  A
// move with dD < 0 bids its packed (dD, C[u]) at best[v] with an atomic
// minimum.  All group reductions are outside the branches, so every lane of
// the warp takes part in every shuffle.
__global__ void __launch_bounds__(kBlock) k_edges(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip) return;
    __shared__ EdgeScratch sh[kWarpsPerBlock];
    const unsigned long long mask = st->mask;
    const int gs = lanes_per_item(a.k), per = 32 / gs;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, l = lane & (gs - 1);
    const unsigned lt = (1u << lane) - 1u;
    const int k = a.k, pad = a.kp - a.k;
    EdgeScratch& es = sh[w];
    const long long nwarps = (long long)gridDim.x * kWarpsPerBlock;
    for (long long base = ((long long)blockIdx.x * kWarpsPerBlock + w) * 32; base < a.nnz; base += nwarps * 32) {
        const long long e = base + lane;
        int v = 0, u = 0, x = -1;
        if (e < a.nnz) {
            v = __ldg(a.src + e);
            u = __ldg(a.col + e);
            if (u != v) {
                x = __ldg(a.C + u);
                if (x == __ldg(a.C + v)) x = -1;
            }
        }
        const unsigned long long pair = x >= 0 ? ((unsigned long long)(unsigned)v << 32) | (unsigned)x : kEmpty;
        const unsigned same = __match_any_sync(kFull, pair);
        const bool keep = x >= 0 && (__ffs(same) - 1) == lane;
        const unsigned km = __ballot_sync(kFull, keep);
        if (keep) {
            const int p = __popc(km & lt);
            const int cv = __ldg(a.C + v);
            es.v[p] = v;
            es.u[p] = u;
            es.x[p] = x;
            es.sx[p] = __ldg(a.size + x);
            es.sa[p] = __ldg(a.size + cv);
            es.Aa[p] = __ldg(a.aown + v);
        }
        __syncwarp();
        const int nf = __popc(km);
        for (int r0 = 0; r0 < nf; r0 += per) {
            const int j = r0 + lane / gs;
            const bool valid = j < nf;
            const int ev = valid ? es.v[j] : 0, eu = valid ? es.u[j] : 0, ex_ = valid ? es.x[j] : 0;
            const int sx = valid ? es.sx[j] : 0, sa = valid ? es.sa[j] : 0, Aa = valid ? es.Aa[j] : 0;
            const bool single = valid && sx == 1;
            const bool table = valid && sx > 1;
            const int* gv = a.G + (long long)ev * a.kp;
            int rc = 0, ex = 0, ub = 0, nq = 0;
            if (single) rc = row_part(a, eu, ev, l, gs);
            if (table) summary_part(a, gv, ex_, l, gs, ex, ub, nq);
            rc = group_sum(rc, gs);
            ex = group_sum(ex, gs);
            ub = group_sum(ub, gs);
            const bool open = table && 2 * (Aa - k - ub) - k * (sa - 1 - sx) < 0;
            int pb = 0;
            if (open) pb = probe_part(a, a.table, mask, gv, ex_, l, gs);
            pb = group_sum(pb, gs);
            if ((single || open) && l == 0) {
                const int A = single ? rc - pad : ex + pb;
                const int dD = 2 * (Aa - k - A) - k * (sa - 1 - sx);
                if (dD < 0) atomicMin(&a.best[ev], pack_key(dD, ex_));
            }
        }
        __syncwarp();
    }
}

// Turns the bids into the proposal list (v, a, b, dD) and clears best[].
// Each block gathers its proposals in shared memory and appends them with one
// global atomic.
__global__ void __launch_bounds__(kBlock) k_collect(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip) return;
    __shared__ int4 sbuf[kBlock];
    __shared__ int s_cnt;
    __shared__ unsigned long long s_base;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long b0 = (long long)blockIdx.x * blockDim.x; b0 < a.n; b0 += stride) {
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        const long long v = b0 + threadIdx.x;
        if (v < a.n) {
            const unsigned long long key = a.best[v];
            if (key != kEmpty) {
                a.best[v] = kEmpty;
                const int p = atomicAdd(&s_cnt, 1);
                sbuf[p] = make_int4((int)v, a.C[v], (int)(unsigned)(key & 0xffffffffull), key_gain(key));
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && s_cnt > 0) s_base = atomicAdd(&st->nprop, (unsigned long long)s_cnt);
        __syncthreads();
        for (int p = threadIdx.x; p < s_cnt; p += blockDim.x) {
            const int4 q = sbuf[p];
            const unsigned long long j = s_base + p;
            a.pv[j] = q.x;
            a.pa[j] = q.y;
            a.pb[j] = q.z;
            a.pg[j] = q.w;
        }
        __syncthreads();
    }
}

// ---- heavy sweeps --------------------------------------------------------
// When a large share of the vertices proposes (|P| > n / 8, or always with
// sweep_mode 2, never with sweep_mode 1), or the table
// does not hold the counts of C yet (the singleton start), dF(P1) is taken
// from a rebuild instead of from staged deltas: P1 is applied to C in place
// (the movers' old clusters stay in the proposal list), the table and its
// summary rows are rebuilt from the new C, and F' - F is dF(P1) exactly.  If
// it is negative, P1 is committed as it stands (mode 3); otherwise the moves
// are undone, the table is rebuilt from C again and the matching fallback
// runs as in a light sweep (mode 2).

__global__ void k_route(SweepArgs a)
{
    DevState* st = a.st;
    st->heavy = 0;
    st->rollback = 0;
    if (st->skip || st->err || st->nprop == 0) return;
    const bool light = a.sweep_mode == 1 || (a.sweep_mode == 0 && st->nprop * 8 <= (unsigned long long)a.n);
    if (st->tvalid && light) return;
    st->heavy = 1;
    st->recompute = 0;
    // keys after applying P1: every vertex gives at most k, every mover at most k new ones
    const unsigned long long kn = (unsigned long long)a.k * a.n;
    unsigned long long bound = (st->tvalid ? (unsigned long long)st->live : kn) + (unsigned long long)a.k * st->nprop;
    if (bound > kn) bound = kn;
    unsigned long long c = a.cap_min;
    while (c < 2 * bound && c < a.mask_max + 1) c <<= 1;
    st->new_mask = c - 1;
    st->rebuild = 1;
}

// Singleton guard on every proposal (sizes of the sweep start); counts |P1|.
__global__ void k_h_mark(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip || !st->heavy) return;
    const long long np = (long long)st->nprop;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < np; base += stride) {
        const long long j = base + threadIdx.x;
        bool keep = false;
        if (j < np) {
            const int ca = a.pa[j], cb = a.pb[j];
            keep = !(a.size[ca] == 1 && a.size[cb] == 1) || cb < ca;
            a.pflag[j] = keep ? 1 : 0;
        }
        const unsigned mk = __ballot_sync(kFull, keep);
        if (lane == 0 && mk) atomicAdd(&st->np1, (unsigned long long)__popc(mk));
    }
}

// Applies (sign +1) or undoes (sign -1) the kept proposals on C and the sizes.
__global__ void k_h_apply(SweepArgs a, int undo)
{
    DevState* st = a.st;
    if (st->skip || !st->heavy || (undo && !st->rollback)) return;
    const long long np = (long long)st->nprop;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < np; j += stride) {
        if (!a.pflag[j]) continue;
        const int ca = a.pa[j], cb = a.pb[j];
        a.C[a.pv[j]] = undo ? ca : cb;
        atomicAdd(&a.size[ca], undo ? 1 : -1);
        atomicAdd(&a.size[cb], undo ? -1 : 1);
    }
}

// F' = k sum_c s_c^2 - 2 sum_keys n^2 (+ sum_ij |P_ij|^2, added in k_h_decide):
// the table part was added by the summary pass of the rebuild, this adds the
// size part.
__global__ void k_h_eval(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip || !st->heavy || st->err) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long b0 = (long long)blockIdx.x * blockDim.x; b0 < a.n; b0 += stride) {
        const long long t = b0 + threadIdx.x;
        long long acc = 0;
        if (t < a.n) {
            const long long sz = a.size[t];
            acc = (long long)a.k * sz * sz;
        }
        block_add64(acc, &st->recompute);
    }
}

__global__ void k_h_decide(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip || !st->heavy) return;
    if (st->err) {
        st->mode = 0;
        return;
    }
    const long long dF = st->recompute + st->partition_sq - st->F;
    st->dF_p1 = st->np1 > 0 ? dF : 0;
    if (st->np1 > 0 && dF < 0) {
        st->mode = 3;
        st->dF = dF;
        st->moves = st->np1;
    } else {
        st->mode = 2;
        st->dF = 0;
        st->moves = 0;
        if (st->np1 > 0) {
            st->rollback = 1;
            st->rebuild = 1;
            st->new_mask = st->mask;
        }
    }
}

// Occupancy above which a sweep is abandoned and retried in a larger table.
__device__ __forceinline__ unsigned long long fill_limit(unsigned long long mask)
{
    return (mask + 1) - ((mask + 1) >> 3);
}

// Adds the warp's new slots to st->used and flags an overflow past the limit.
__device__ __forceinline__ void count_inserts(DevState* st, unsigned mi, unsigned long long mask)
{
    if (mi) {
        const unsigned long long old = atomicAdd(&st->used, (unsigned long long)__popc(mi));
        if (old + __popc(mi) > fill_limit(mask)) st->overflow = 1;
    }
}

// One thread per (proposal j, partition i).  Staging never fails: if the
// table runs short of slots the sweep is abandoned (st->overflow) before
// anything is committed, and k_end schedules a larger table and a retry.
__global__ void k_stage(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip || st->err || st->heavy) return;
    const unsigned long long mask = st->mask;
    const long long total = (long long)st->nprop * a.k;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < total; base += stride) {
        const long long t = base + threadIdx.x;
        bool ins = false, head = false;
        if (t < total) {
            const long long j = t / a.k;
            const int i = (int)(t - j * a.k);
            const int v = a.pv[j], ca = a.pa[j], cb = a.pb[j];
            const bool keep = !(a.size[ca] == 1 && a.size[cb] == 1) || cb < ca;
            if (i == 0) {
                a.pflag[j] = keep ? 1 : 0;
                if (keep) {
                    atomicAdd(&a.dsize[ca], -1);
                    atomicAdd(&a.dsize[cb], 1);
                    head = true;
                }
            }
            if (keep) {
                const int g = a.G[(long long)v * a.kp + i];
                const long long sa = table_find(a.table, mask, ckey(ca, g));
                const long long sb = table_find_or_insert(a.table, mask, ckey(cb, g), &ins);
                if (sa < 0) {
                    set_err(st, CC_ERR_INVALID);  // the vertex's own key must exist
                } else if (sb < 0) {
                    st->overflow = 1;
                } else {
                    atomicAdd(&a.table[sa].dlt, -1);
                    atomicAdd(&a.table[sb].dlt, 1);
                    a.pslot[2 * t] = (unsigned)sa;
                    a.pslot[2 * t + 1] = (unsigned)sb;
                }
            }
        }
        const unsigned mi = __ballot_sync(kFull, ins), mh = __ballot_sync(kFull, head);
        if (lane == 0) {
            count_inserts(st, mi, mask);
            if (mh) atomicAdd(&st->np1, (unsigned long long)__popc(mh));
        }
    }
}

// dF(P1) = k sum_c ((s+ds)^2 - s^2) - 2 sum_keys ((n+dn)^2 - n^2), written as a
// sum over the staged contributions: each +-1 added to an entry x with final
// delta d_x contributes +-(2 x + d_x).
__global__ void k_eval(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip || st->err || st->overflow || st->heavy) return;
    const long long total = (long long)st->nprop * a.k;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < total; base += stride) {
        const long long t = base + threadIdx.x;
        long long acc = 0;
        if (t < total) {
            const long long j = t / a.k;
            const int i = (int)(t - j * a.k);
            if (a.pflag[j]) {
                const ulonglong2 A = *reinterpret_cast<const ulonglong2*>(a.table + a.pslot[2 * t]);
                const ulonglong2 B = *reinterpret_cast<const ulonglong2*>(a.table + a.pslot[2 * t + 1]);
                const long long an = (int)(unsigned)(A.y & 0xffffffffull), ad = (int)(unsigned)(A.y >> 32);
                const long long bn = (int)(unsigned)(B.y & 0xffffffffull), bd = (int)(unsigned)(B.y >> 32);
                acc = -2 * (-(2 * an + ad) + (2 * bn + bd));
                if (i == 0) {
                    const int ca = a.pa[j], cb = a.pb[j];
                    acc += (long long)a.k * (-(2LL * a.size[ca] + a.dsize[ca]) + (2LL * a.size[cb] + a.dsize[cb]));
                }
            }
        }
        block_add64(acc, &st->dF);
    }
}

__global__ void k_decide(DevState* st)
{
    if (st->skip || st->heavy) return;
    if (st->err || st->overflow) {
        st->mode = 0;
        return;
    }
    if (st->np1 > 0 && st->dF < 0) {
        st->mode = 1;
        st->dF_p1 = st->dF;
        st->moves = st->np1;
    } else if (st->nprop > 0) {
        st->mode = 2;
        st->dF_p1 = st->np1 > 0 ? st->dF : 0;
        st->dF = 0;
        st->moves = 0;
    } else {
        st->mode = 0;
        st->dF = 0;
    }
}

__global__ void k_commit(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip || st->err) return;
    const int mode = st->mode;
    if (mode == 0 || mode == 3) return;
    const bool staged = !st->heavy;  // only light sweeps staged deltas to undo
    const long long total = (long long)st->nprop * a.k;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < total; base += stride) {
        const long long t = base + threadIdx.x;
        long long live = 0;
        if (t < total) {
            const long long j = t / a.k;
            const int i = (int)(t - j * a.k);
            const int ca = a.pa[j], cb = a.pb[j];
            if (mode == 1) {
                if (a.pflag[j]) {
                    if (i == 0) {
                        a.C[a.pv[j]] = cb;
                        int d = atomicExch(&a.dsize[ca], 0);
                        if (d) atomicAdd(&a.size[ca], d);
                        d = atomicExch(&a.dsize[cb], 0);
                        if (d) atomicAdd(&a.size[cb], d);
                    }
#pragma unroll
                    for (int side = 0; side < 2; ++side) {
                        Slot* s = a.table + a.pslot[2 * t + side];
                        const int d = atomicExch(&s->dlt, 0);
                        if (d) {
                            const int old = atomicAdd(&s->cnt, d);
                            live += (old == 0) - (old + d == 0);
                            summ_update(a.summ, a.kp, a.lshift, s->key, d, old + d);
                        }
                    }
                }
            } else {
                if (staged && a.pflag[j]) {
                    a.table[a.pslot[2 * t]].dlt = 0;
                    a.table[a.pslot[2 * t + 1]].dlt = 0;
                    if (i == 0) {
                        a.dsize[ca] = 0;
                        a.dsize[cb] = 0;
                    }
                }
                if (i == 0) {
                    const unsigned long long key = pack_key(a.pg[j], a.pv[j]);
                    atomicMin(&a.best[ca], key);
                    atomicMin(&a.best[cb], key);
                }
            }
        }
        block_add64(live, &st->live);
    }
}

// Fallback: a proposal is committed iff its (dD, v) is the least at both of
// its clusters; the committed moves touch pairwise-disjoint clusters, so
// their objective changes add exactly.  Phase 1 (thread per (proposal,
// partition)) marks the winners and inserts their target keys, so that an
// overflow is seen before any count changes; phase 2 applies the moves.
__global__ void k_match_keys(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip || st->err || st->mode != 2) return;
    const unsigned long long mask = st->mask;
    const long long total = (long long)st->nprop * a.k;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < total; base += stride) {
        const long long t = base + threadIdx.x;
        bool ins = false;
        if (t < total) {
            const long long j = t / a.k;
            const int i = (int)(t - j * a.k);
            const int v = a.pv[j], ca = a.pa[j], cb = a.pb[j];
            const unsigned long long key = pack_key(a.pg[j], v);
            if (a.best[ca] == key && a.best[cb] == key) {
                if (i == 0) a.pflag[j] = 2;
                const long long sb = table_find_or_insert(a.table, mask, ckey(cb, a.G[(long long)v * a.kp + i]), &ins);
                if (sb < 0) st->overflow = 1;
            }
        }
        const unsigned mi = __ballot_sync(kFull, ins);
        if (lane == 0) count_inserts(st, mi, mask);
    }
}

__global__ void k_match_apply(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip || st->err || st->overflow || st->mode != 2) return;
    const unsigned long long mask = st->mask;
    const long long total = (long long)st->nprop * a.k;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < total; base += stride) {
        const long long t = base + threadIdx.x;
        long long live = 0;
        if (t < total) {
            const long long j = t / a.k;
            const int i = (int)(t - j * a.k);
            if (a.pflag[j] == 2) {
                const int v = a.pv[j], ca = a.pa[j], cb = a.pb[j];
                if (i == 0) {
                    a.C[v] = cb;
                    atomicAdd(&a.size[ca], -1);
                    atomicAdd(&a.size[cb], 1);
                    atomicAdd(&st->moves, 1ull);
                    atomicAdd(reinterpret_cast<unsigned long long*>(&st->dF), (unsigned long long)(2LL * a.pg[j]));
                }
                const int g = a.G[(long long)v * a.kp + i];
                const long long sa = table_find(a.table, mask, ckey(ca, g));
                const long long sb = table_find(a.table, mask, ckey(cb, g));
                if (sa < 0 || sb < 0) {
                    set_err(st, CC_ERR_INVALID);
                } else {
                    const int oa = atomicAdd(&a.table[sa].cnt, -1);
                    const int ob = atomicAdd(&a.table[sb].cnt, 1);
                    live += (ob == 0) - (oa == 1);
                    summ_update(a.summ, a.kp, a.lshift, ckey(ca, g), -1, oa - 1);
                    summ_update(a.summ, a.kp, a.lshift, ckey(cb, g), 1, ob + 1);
                }
            }
        }
        block_add64(live, &st->live);
    }
}

__global__ void k_match_reset(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip || st->mode != 2) return;
    const long long np = (long long)st->nprop;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < np; j += stride) {
        a.best[a.pa[j]] = kEmpty;
        a.best[a.pb[j]] = kEmpty;
    }
}

__global__ void k_end(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip) return;
    if (st->err) {
        st->stop = 1;
        return;
    }
    const unsigned long long cap = st->mask + 1;
    if (st->overflow) {
        // nothing was committed: retry this sweep after rebuilding into twice
        // the capacity (the staged deltas are discarded with the old table)
        if (cap >= a.mask_max + 1) {
            set_err(st, CC_ERR_TABLE_FULL);
            st->stop = 1;
            return;
        }
        st->new_mask = 2 * cap - 1;
        st->abort = 1;
        st->rebuild = 1;
        st->retries += 1;
        return;
    }
    if (st->mode != 0) st->F += st->dF;
    if (st->sweeps < a.hist_cap) {
        cc_sweep_info r;
        r.proposals = (int64_t)st->nprop;
        r.p1 = (int64_t)st->np1;
        r.dF_p1 = st->dF_p1;
        r.fallback = st->mode == 2 ? 1 : 0;
        r.moves = (int64_t)st->moves;
        r.F = st->F;
        a.hist[st->sweeps] = r;
    }
    st->sweeps += 1;
    st->run_sweeps += 1;
    if (st->nprop == 0 || st->run_sweeps >= st->run_limit) st->stop = 1;
    // compaction: rebuild without the dead keys when occupied slots pass one
    // half of the capacity; the new capacity holds the live keys plus k x
    // (moves of this sweep), a forecast of the next sweep's new keys, at load
    // <= 1/2.  (Summary rows settle most of each score, so a table larger than
    // needed costs little; it is not shrunk otherwise.)
    const unsigned long long live = (unsigned long long)st->live;
    const unsigned long long want = 2 * (live + (unsigned long long)a.k * st->moves);
    unsigned long long c = a.cap_min;
    while (c < want && c < a.mask_max + 1) c <<= 1;
    if (st->tvalid && st->used > cap / 2) {
        st->new_mask = c - 1;
        st->rebuild = 1;
    } else {
        st->rebuild = 0;
    }
}

}  // namespace

cudaError_t prepare_propose(int kp, int* blocks_per_sm)
{
    (void)kp;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_edges, kBlock, 0);
}

cudaError_t launch_run_begin(DevState* st, int limit, cudaStream_t s)
{
    k_run_begin<<<1, 1, 0, s>>>(st, limit);
    return cudaGetLastError();
}

cudaError_t launch_sweep(const SweepArgs& a, int grid, cudaStream_t s, cudaEvent_t prop0, cudaEvent_t prop1)
{
    const int g2 = grid;
    k_begin<<<1, 1, 0, s>>>(a.st);
    if (prop0) {
        cudaError_t e = cudaEventRecordWithFlags(prop0, s, cudaEventRecordExternal);
        if (e != cudaSuccess) return e;
    }
    k_own<<<grid, kBlock, 0, s>>>(a);
    k_edges<<<grid, kBlock, 0, s>>>(a);
    k_collect<<<grid, kBlock, 0, s>>>(a);
    if (prop1) {
        cudaError_t e = cudaEventRecordWithFlags(prop1, s, cudaEventRecordExternal);
        if (e != cudaSuccess) return e;
    }
    k_route<<<1, 1, 0, s>>>(a);
    k_h_mark<<<g2, kBlock, 0, s>>>(a);
    k_h_apply<<<g2, kBlock, 0, s>>>(a, 0);
    {
        cudaError_t e = launch_table_rebuild(a, true, s);
        if (e != cudaSuccess) return e;
    }
    k_h_eval<<<g2, kBlock, 0, s>>>(a);
    k_h_decide<<<1, 1, 0, s>>>(a);
    k_h_apply<<<g2, kBlock, 0, s>>>(a, 1);
    {
        cudaError_t e = launch_table_rebuild(a, true, s);
        if (e != cudaSuccess) return e;
    }
    k_stage<<<g2, kBlock, 0, s>>>(a);
    k_eval<<<g2, kBlock, 0, s>>>(a);
    k_decide<<<1, 1, 0, s>>>(a.st);
    k_commit<<<g2, kBlock, 0, s>>>(a);
    k_match_keys<<<g2, kBlock, 0, s>>>(a);
    k_match_apply<<<g2, kBlock, 0, s>>>(a);
    k_match_reset<<<g2, kBlock, 0, s>>>(a);
    k_end<<<1, 1, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_table_rebuild(a, true, s);
}

}  // namespace ccg
