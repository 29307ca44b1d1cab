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

// A_x = sum_i n(x, g_i(v)) by k probes, four first loads in flight at a time.
__device__ __forceinline__ int agree_table(const Slot* __restrict__ t, unsigned long long mask, int x,
                                           const int* sg, int k)
{
    int A = 0;
    int i = 0;
    for (; i + 4 <= k; i += 4) {
        const unsigned long long k0 = ckey(x, sg[i]), k1 = ckey(x, sg[i + 1]);
        const unsigned long long k2 = ckey(x, sg[i + 2]), k3 = ckey(x, sg[i + 3]);
        const unsigned long long h0 = mix64(k0) & mask, h1 = mix64(k1) & mask;
        const unsigned long long h2 = mix64(k2) & mask, h3 = mix64(k3) & mask;
        const ulonglong2 e0 = __ldg(reinterpret_cast<const ulonglong2*>(t + h0));
        const ulonglong2 e1 = __ldg(reinterpret_cast<const ulonglong2*>(t + h1));
        const ulonglong2 e2 = __ldg(reinterpret_cast<const ulonglong2*>(t + h2));
        const ulonglong2 e3 = __ldg(reinterpret_cast<const ulonglong2*>(t + h3));
        A += resolve(t, mask, k0, h0, e0) + resolve(t, mask, k1, h1, e1) + resolve(t, mask, k2, h2, e2) +
             resolve(t, mask, k3, h3, e3);
    }
    for (; i < k; ++i) A += table_count_ro(t, mask, ckey(x, sg[i]));
    return A;
}

// Partitions in which u agrees with v: u's label row (16-byte aligned, kp
// entries, padding -1) against v's row in shared memory (padding -2).
__device__ __forceinline__ int agree_row(const int* __restrict__ gu, const int* sg, int kp)
{
    const int4* g4 = reinterpret_cast<const int4*>(gu);
    const int4* s4 = reinterpret_cast<const int4*>(sg);
    int A = 0;
    for (int q = 0; q < (kp >> 2); ++q) {
        const int4 a = __ldg(g4 + q);
        const int4 b = s4[q];
        A += (a.x == b.x) + (a.y == b.y) + (a.z == b.z) + (a.w == b.w);
    }
    return A;
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
    st->nprop = 0;
    st->np1 = 0;
    st->dF = 0;
    st->dF_p1 = 0;
    st->moves = 0;
    st->tile_ctr = 0;
    st->mode = 0;
}

// Warp per vertex; each lane takes one neighbour of a 32-wide chunk, equal
// candidate clusters inside the chunk are merged with __match_any_sync, and
// every distinct candidate is scored by the lane that holds it.  Blocks claim
// tiles of kTile vertices and their warps claim single vertices from the
// tile, which balances skewed degrees; proposals are gathered per tile in
// shared memory and appended with one global atomic.
__global__ void __launch_bounds__(kBlock) k_propose(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip) return;
    extern __shared__ int4 smem4[];
    int4* sbuf = smem4;                                   // kTile proposals
    int* sG = reinterpret_cast<int*>(smem4 + kTile);       // own label row per warp
    __shared__ long long s_tile;
    __shared__ int s_next, s_cnt;
    __shared__ unsigned long long s_gbase;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int* sg = sG + w * a.kp;
    const int k = a.k;

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
            const int cv = __ldg(a.C + v);
            const int sa = __ldg(a.size + cv);
            const int* gv = a.G + (long long)v * a.kp;
            for (int i = lane; i < a.kp; i += 32) sg[i] = i < k ? __ldg(gv + i) : -2;
            __syncwarp();
            int Aa = k;
            if (sa > 1) {
                int part = 0;
                for (int i = lane; i < k; i += 32) part += table_count_ro(a.table, a.mask, ckey(cv, sg[i]));
                Aa = __reduce_add_sync(kFull, part);
            }
            unsigned long long best = kEmpty;
            const long long beg = __ldg(a.off + v), end = __ldg(a.off + v + 1);
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
                if (x >= 0 && (__ffs(m) - 1) == lane) {
                    const int sx = __ldg(a.size + x);
                    const int Ax = sx == 1 ? agree_row(a.G + (long long)u * a.kp, sg, a.kp)
                                           : agree_table(a.table, a.mask, x, sg, k);
                    const int dD = 2 * (Aa - k - Ax) - k * (sa - 1 - sx);
                    const unsigned long long key = pack_key(dD, x);
                    best = key < best ? key : best;
                }
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

// One thread per (proposal j, partition i).
__global__ void k_stage(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip || st->err) return;
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
                const long long sa = table_find(a.table, a.mask, ckey(ca, g));
                const long long sb = table_find_or_insert(a.table, a.mask, ckey(cb, g), &ins);
                if (sa < 0) {
                    set_err(st, CC_ERR_INVALID);  // the vertex's own key must exist
                } else if (sb < 0) {
                    set_err(st, CC_ERR_TABLE_FULL);
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
            if (mi) atomicAdd(&st->used, (unsigned long long)__popc(mi));
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
    if (st->skip || st->err) return;
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
    if (st->err) {
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
// their objective changes add exactly.
__global__ void k_match_commit(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip || st->err || st->mode != 2) return;
    const long long np = (long long)st->nprop;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < np; j += stride) {
        const int v = a.pv[j], ca = a.pa[j], cb = a.pb[j], g = a.pg[j];
        const unsigned long long key = pack_key(g, v);
        if (a.best[ca] != key || a.best[cb] != key) continue;
        a.C[v] = cb;
        atomicAdd(&a.size[ca], -1);
        atomicAdd(&a.size[cb], 1);
        long long live = 0;
        unsigned long long used = 0;
        for (int i = 0; i < a.k; ++i) {
            const int gg = a.G[(long long)v * a.kp + i];
            const long long sa = table_find(a.table, a.mask, ckey(ca, gg));
            bool ins = false;
            const long long sb = table_find_or_insert(a.table, a.mask, ckey(cb, gg), &ins);
            if (sa < 0) { set_err(st, CC_ERR_INVALID); continue; }
            if (sb < 0) { set_err(st, CC_ERR_TABLE_FULL); continue; }
            used += ins;
            if (atomicAdd(&a.table[sa].cnt, -1) == 1) --live;
            if (atomicAdd(&a.table[sb].cnt, 1) == 0) ++live;
        }
        if (live) atomicAdd(reinterpret_cast<unsigned long long*>(&st->live), (unsigned long long)live);
        if (used) atomicAdd(&st->used, used);
        atomicAdd(&st->moves, 1ull);
        atomicAdd(reinterpret_cast<unsigned long long*>(&st->dF), (unsigned long long)(2LL * g));
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
    st->rebuild = st->used > a.thresh ? 1 : 0;
}

}  // namespace

size_t propose_smem_bytes(int kp)
{
    return sizeof(int4) * kTile + sizeof(int) * (size_t)kWarpsPerBlock * kp;
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
    k_match_commit<<<g2, kBlock, 0, s>>>(a);
    k_match_reset<<<g2, kBlock, 0, s>>>(a);
    k_end<<<1, 1, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_table_rebuild(a, true, s);
}

}  // namespace ccg
