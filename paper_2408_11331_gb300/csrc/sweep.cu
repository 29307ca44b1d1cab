// One synchronous local-move sweep (Methods, "Parallel algorithm"), as a fixed
// sequence of kernels on one stream so that it can be captured in a CUDA graph:
//
//   begin       per-sweep counters; the sweep is skipped once the run has stopped
//   propose     best move of every vertex against the sweep-start state
//               (Eq. objective4 with the gain of Eq. objective3)
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

__device__ __forceinline__ unsigned long long warp_min64(unsigned long long x)
{
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long y = __shfl_xor_sync(kFull, x, o);
        x = y < x ? y : x;
    }
    return x;
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

// Per-warp scratch of the proposal kernel (shared memory).
struct WarpScratch {
    int cx[33];    // entries to score: the own cluster (entry 0, when not a singleton), then
    int cu[33];    // the distinct candidate clusters of the chunk, a neighbour carrying each
    int cs[33];    // (the only member for a singleton), and their sizes
    int seen[128]; // candidates already scored for this vertex (degree > 32 only)
};

constexpr int kInflight = 4;  // table probes per lane issued before the first is resolved

// Agreement A_x = sum_i n(x, g_i(v)) of the entry held by this lane's group:
// the warp is split into groups of gs lanes (gs = 32 / next_pow2(entries)), one
// entry per group; the lanes of a group share the partitions.  A singleton {u}
// is scored from u's label row against v's (int4 loads), any other cluster by
// hash probes with kInflight first loads in flight per lane.  The group's
// lanes are summed with xor shuffles (groups are aligned, so they stay apart).
__device__ __forceinline__ int score_entry(const SweepArgs& a, const Slot* __restrict__ table,
                                           unsigned long long mask, const int* sg, int x, int u, int sx,
                                           bool valid, int l, int gs)
{
    int acc = 0;
    if (valid) {
        if (sx == 1) {
            const int4* g4 = reinterpret_cast<const int4*>(a.G + (long long)u * a.kp);
            const int4* s4 = reinterpret_cast<const int4*>(sg);
            const int kq = a.kp >> 2;
            for (int q0 = l; q0 < kq; q0 += gs * 8) {
                int4 r[8];
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    const int q = q0 + b * gs;
                    r[b] = q < kq ? __ldg(g4 + q) : make_int4(-1, -1, -1, -1);
                }
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    const int q = q0 + b * gs;
                    if (q < kq) {
                        const int4 s = s4[q];
                        acc += (r[b].x == s.x) + (r[b].y == s.y) + (r[b].z == s.z) + (r[b].w == s.w);
                    }
                }
            }
        } else {
            for (int i0 = l; i0 < a.k; i0 += gs * kInflight) {
                unsigned long long key[kInflight], h[kInflight];
                ulonglong2 ev[kInflight];
#pragma unroll
                for (int b = 0; b < kInflight; ++b) {
                    const int i = i0 + b * gs;
                    key[b] = 0;
                    h[b] = 0;
                    ev[b] = make_ulonglong2(kEmpty, 0ull);
                    if (i < a.k) {
                        key[b] = ckey(x, sg[i]);
                        h[b] = mix64(key[b]) & mask;
                        ev[b] = __ldg(reinterpret_cast<const ulonglong2*>(table + h[b]));
                    }
                }
#pragma unroll
                for (int b = 0; b < kInflight; ++b)
                    if (i0 + b * gs < a.k) acc += resolve(table, mask, key[b], h[b], ev[b]);
            }
        }
    }
    for (int o = gs >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    return acc;
}

// Warp per vertex.  Each chunk of 32 neighbours: the lane holding a neighbour
// reads its cluster; equal clusters are merged with __match_any_sync (and,
// past the first chunk, with a per-warp seen-set) and the distinct candidates
// are compacted into shared memory, after the vertex's own cluster in the
// first chunk.  The warp then scores all entries at once, one group of lanes
// per entry (score_entry), and keeps the least packed (dD, id).  Blocks claim
// 256-vertex tiles and warps claim single vertices from their tile, which
// balances skewed degrees; proposals are gathered per tile in shared memory
// and appended with one global atomic per tile.
__global__ void __launch_bounds__(kBlock) k_propose(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip) return;
    const unsigned long long mask = st->mask;
    extern __shared__ int4 smem4[];
    int4* sbuf = smem4;                                            // kTile proposals
    WarpScratch* wsall = reinterpret_cast<WarpScratch*>(smem4 + kTile);
    int* sG = reinterpret_cast<int*>(wsall + kWarpsPerBlock);      // own label row per warp
    __shared__ long long s_tile;
    __shared__ int s_next, s_cnt;
    __shared__ unsigned long long s_gbase;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    WarpScratch& ws = wsall[w];
    int* sg = sG + w * a.kp;
    const int k = a.k;
    const Slot* __restrict__ table = a.table;

    for (;;) {
        if (threadIdx.x == 0) {
            s_tile = (long long)atomicAdd(&st->tile_ctr, (unsigned long long)kTile);
            s_next = 0;
            s_cnt = 0;
        }
        __syncthreads();
        const long long tile = s_tile;
        if (tile >= a.n) break;
        const int tlen = (int)min((long long)kTile, (long long)a.n - tile);
        for (;;) {
            int idx = 0;
            if (lane == 0) idx = atomicAdd(&s_next, 1);
            idx = __shfl_sync(kFull, idx, 0);
            if (idx >= tlen) break;
            const int v = (int)(tile + idx);
            const long long beg = __ldg(a.off + v), end = __ldg(a.off + v + 1);
            if (beg == end) continue;  // isolated: never moves
            const int cv = __ldg(a.C + v);
            const int sa = __ldg(a.size + cv);
            const int* gv = a.G + (long long)v * a.kp;
            for (int i = lane; i < a.kp; i += 32) sg[i] = i < k ? __ldg(gv + i) : -2;
            const bool use_seen = end - beg > 32;
            if (use_seen)
                for (int q = lane; q < 128; q += 32) ws.seen[q] = -1;
            __syncwarp();
            int Aa = k;  // A_a = sum_i n(a, g_i(v)); k for a singleton
            unsigned long long best = kEmpty;
            for (long long base = beg; base < end; base += 32) {
                const long long e = base + lane;
                int u = -1, x = -1;
                if (e < end) {
                    u = __ldg(a.col + e);
                    if (u != v) {
                        x = __ldg(a.C + u);
                        if (x == cv) x = -1;
                    }
                }
                const unsigned m = __match_any_sync(kFull, x);
                bool lead = x >= 0 && (__ffs(m) - 1) == lane;
                if (use_seen && lead) {
                    unsigned h = ((unsigned)x * 2654435761u) >> 25;
                    for (int t = 0; t < 128; ++t, h = (h + 1) & 127) {
                        const int old = atomicCAS(&ws.seen[h], -1, x);
                        if (old == -1) break;
                        if (old == x) { lead = false; break; }
                    }
                }
                const bool own = base == beg && sa > 1;  // the own cluster is scored with the first chunk
                const int e0 = own ? 1 : 0;
                const unsigned lb = __ballot_sync(kFull, lead);
                const int ne = e0 + __popc(lb);
                if (lane == 0 && own) {
                    ws.cx[0] = cv;
                    ws.cu[0] = v;
                    ws.cs[0] = sa;
                }
                if (lead) {
                    const int p = e0 + __popc(lb & lt);
                    ws.cx[p] = x;
                    ws.cu[p] = u;
                    ws.cs[p] = __ldg(a.size + x);
                }
                __syncwarp();
                // groups of gs lanes, 32 / gs >= entries (33 entries: two passes of 32)
                for (int p0 = 0; p0 < ne; p0 += 32) {
                    const int cnt = min(32, ne - p0);
                    const int gs = cnt > 16 ? 1 : cnt > 8 ? 2 : cnt > 4 ? 4 : cnt > 2 ? 8 : cnt > 1 ? 16 : 32;
                    const int j = p0 + lane / gs, l = lane & (gs - 1);
                    const bool valid = j < ne;
                    const int xj = valid ? ws.cx[j] : 0, uj = valid ? ws.cu[j] : 0, sj = valid ? ws.cs[j] : 0;
                    const int A = score_entry(a, table, mask, sg, xj, uj, sj, valid, l, gs);
                    if (own && p0 == 0) Aa = __shfl_sync(kFull, A, 0);
                    if (valid && l == 0 && !(own && j == 0)) {
                        const int dD = 2 * (Aa - k - A) - k * (sa - 1 - sj);
                        const unsigned long long kk = pack_key(dD, xj);
                        best = kk < best ? kk : best;
                    }
                }
                __syncwarp();
            }
            best = warp_min64(best);
            if (lane == 0 && best != kEmpty && key_gain(best) < 0) {
                const int p = atomicAdd(&s_cnt, 1);
                sbuf[p] = make_int4(v, cv, (int)(unsigned)(best & 0xffffffffull), key_gain(best));
            }
            __syncwarp();
        }
        __syncthreads();
        if (threadIdx.x == 0 && s_cnt > 0) s_gbase = atomicAdd(&st->nprop, (unsigned long long)s_cnt);
        __syncthreads();
        for (int p = threadIdx.x; p < s_cnt; p += blockDim.x) {
            const int4 e = sbuf[p];
            const unsigned long long j = s_gbase + p;
            a.pv[j] = e.x;
            a.pa[j] = e.y;
            a.pb[j] = e.z;
            a.pg[j] = e.w;
        }
        __syncthreads();
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
    if (st->skip || st->err) return;
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
    if (st->skip || st->err || st->overflow) return;
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
    if (st->skip) return;
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
    if (mode == 0) return;
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
                        }
                    }
                }
            } else {
                if (a.pflag[j]) {
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
                    if (atomicAdd(&a.table[sa].cnt, -1) == 1) --live;
                    if (atomicAdd(&a.table[sb].cnt, 1) == 0) ++live;
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
    // compaction: rebuild when occupied slots pass one half (dead keys), or
    // shrink when the live keys fill less than one sixth of the capacity.  The
    // new capacity holds the live keys plus half of k x (moves of this sweep),
    // a forecast of the next sweep's new keys, at load <= 1/2.
    const unsigned long long live = (unsigned long long)st->live;
    const unsigned long long want = 2 * live + (unsigned long long)a.k * st->moves;
    unsigned long long c = a.cap_min;
    while (c < want && c < a.mask_max + 1) c <<= 1;
    if (st->used > cap / 2 || (live * 6 < cap && c < cap)) {
        st->new_mask = c - 1;
        st->rebuild = 1;
    } else {
        st->rebuild = 0;
    }
}

}  // namespace

size_t propose_smem_bytes(int kp)
{
    return sizeof(int4) * kTile + sizeof(WarpScratch) * kWarpsPerBlock + sizeof(int) * (size_t)kWarpsPerBlock * kp;
}

cudaError_t prepare_propose(int kp, int* blocks_per_sm)
{
    const size_t smem = propose_smem_bytes(kp);
    cudaError_t e = cudaFuncSetAttribute(k_propose, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_propose, kBlock, smem);
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
    k_propose<<<grid, kBlock, propose_smem_bytes(a.kp), s>>>(a);
    if (prop1) {
        cudaError_t e = cudaEventRecordWithFlags(prop1, s, cudaEventRecordExternal);
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
