// One synchronous local-move sweep (Methods, "Parallel algorithm") of every
// job of a context, as a fixed sequence of kernels on one stream so that it
// can be captured in a CUDA graph:
//
//   begin        per-sweep counters (union-wide and per job), the sweep's
//                stamp; the sweep is skipped once every job has stopped
//   own/edges/   best move of every vertex against the sweep-start state
//   collect      (Eq. objective4 with the gain of Eq. objective3): A_a per
//                vertex whose cluster changed, then lane groups scoring the
//                distinct candidates of every 128 CSR entries and bidding,
//                then the proposal list
//   route        heavy or light evaluation of the kept moves P1 (results agree)
//   [heavy path] apply P1, rebuild the table (first at a tight capacity, and
//                again at a safe one if the keys did not fit), F' - F per
//                job; commit, or
//   [rollback]   undo and rebuild
//   [light path] singleton guard; stage size and count deltas; exact dF per job
//   bid          matching jobs: drop staged deltas, bid (dD, v) at both clusters
//   match_keys   winners (least (dD, v) at both ends) insert their target keys
//   commit       fold staged deltas in (light P1), move the matching winners;
//                every move stamps its two clusters
//   end          objective, history, stop per job; retry / compaction decisions
//   [rebuild]    rebuild of the contingency hash when one is pending
//
// The bracketed parts are IF regions of the captured graph, entered only when
// a one-thread gate kernel finds them needed (all their kernels also check
// the control block, so a graph without regions gives the same results).
//
// Gain of v moving from its cluster a to b (Eq. objective3, u = v excluded),
// with k the number of partitions of v's job:
//   dD = 2 (A_a - k - A_b) - k (|a| - 1 - |b|),   A_x = sum_i n(x, i, l_i(v)),
// and the move changes the job's F by 2 dD.
#include "context.cuh"

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

// Adds the warp's sum of x to *out (one atomic).  All lanes must call it.
__device__ __forceinline__ void warp_add64(long long x, long long* out)
{
    x = warp_sum64(x);
    if ((threadIdx.x & 31) == 0 && x != 0) atomicAdd(reinterpret_cast<unsigned long long*>(out), (unsigned long long)x);
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

__global__ void k_run_begin(SweepArgs a, int limit)
{
    DevState* st = a.st;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->stop = 0;
        st->run_limit = limit;
        st->run_bodies = 0;
        st->all_active = 1;
        st->cls = 0;
    }
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < a.jobs; j += gridDim.x * blockDim.x) {
        a.js[j].stop = 0;
        a.js[j].run_sweeps = 0;
    }
}

__global__ void k_begin(SweepArgs a)
{
    DevState* st = a.st;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->skip = (st->stop || st->err) ? 1 : 0;
        if (!st->skip) st->stamp += 1;
        st->nprop = 0;
        st->pkeys = 0;
        st->overflow = 0;
        st->heavy = 0;
        st->rollback = 0;
        st->active = 0;
        st->tight = 0;
        st->again = 0;
        st->build_fail = 0;
    }
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < a.jobs; j += gridDim.x * blockDim.x) {
        JobState& s = a.js[j];
        s.nprop = 0;
        s.np1 = 0;
        s.moves = 0;
        s.dF = 0;
        s.dF_p1 = 0;
        s.mode = 0;
        s.rollback = 0;
        s.recompute = 0;
    }
}

constexpr int kInflight = 2;  // loads per lane issued before the first is used

__device__ __forceinline__ int group_sum(int x, int gs)
{
    for (int o = gs >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

// The partitions of a job are scored four at a time ("quads"): partition
// 4q + t is component t of quad q of v's label row (one int4 load) and entry
// 4q + t of x's summary row (one int4 {d1, m1, d2, m2} per partition).  Rows
// are kp = k rounded up to 4 entries, so only the last quad can hold padding,
// which is masked out (4q + t >= k).  Lane l of a group takes quads l,
// l + gs, ...

// Adds one partition to the summary sums: v's label g against the entry e =
// {d1, m1, d2, m2} of a cluster of size sx.
__device__ __forceinline__ void summary_one(int g, int4 e, bool on, int sx, int& ex, int& ub)
{
    if (!on) return;
    const int m = g == e.x ? e.y : (g == e.z ? e.w : 0);
    ex += m;
    // a label other than d1, d2 has at most sx - m1 - m2 members (none when
    // the two cover the cluster)
    ub += (g == e.x || g == e.z) ? m : sx - e.y - e.w;
}

// Summary part of A_x(v) for a non-singleton cluster x (size sx) of job J:
// ex = the counts of v's labels where they are one of the row's two labels
// (exact there; 0, also exact, where the two cover the cluster), ub = ex +
// sum of (sx - m1 - m2) over the other partitions, an upper bound on A_x.
__device__ __forceinline__ void summary_part(const SweepArgs& a, const JobInfo& J, const int* __restrict__ gv, int x,
                                             int sx, int l, int gs, int& ex, int& ub)
{
    ex = 0;
    ub = 0;
    const int4* G4 = reinterpret_cast<const int4*>(gv);
    const int4* S4 = a.summ + row_of(J, x);
    const int kq = J.kp >> 2, k = J.k;
    for (int q = l; q < kq; q += gs) {
        const int4 g = __ldg(G4 + q);
        const int4 e0 = __ldg(S4 + 4 * q), e1 = __ldg(S4 + 4 * q + 1), e2 = __ldg(S4 + 4 * q + 2),
                   e3 = __ldg(S4 + 4 * q + 3);
        const int i = 4 * q;
        summary_one(g.x, e0, i < k, sx, ex, ub);
        summary_one(g.y, e1, i + 1 < k, sx, ex, ub);
        summary_one(g.z, e2, i + 2 < k, sx, ex, ub);
        summary_one(g.w, e3, i + 3 < k, sx, ex, ub);
    }
}

// Starts the probe of one partition if the summary leaves it open (v carries
// neither of the row's labels and the two do not cover x): the key, its
// first slot and that slot's contents.
__device__ __forceinline__ bool probe_start(const Slot* __restrict__ table, unsigned long long mask, int x, int g,
                                            int4 e, bool on, int sx, unsigned long long& key, unsigned long long& h,
                                            ulonglong2& ev)
{
    if (!on || g == e.x || g == e.z || sx <= e.y + e.w) return false;
    key = ckey(x, g);
    h = hash_key(key) & mask;
    ev = __ldg(reinterpret_cast<const ulonglong2*>(table + h));
    return true;
}

// Exact counts of the partitions the summary leaves open, by hash probes
// (four in flight per lane).
__device__ __forceinline__ int probe_part(const SweepArgs& a, const JobInfo& J, const Slot* __restrict__ table,
                                          unsigned long long mask, const int* __restrict__ gv, int x, int sx, int l,
                                          int gs)
{
    const int4* G4 = reinterpret_cast<const int4*>(gv);
    const int4* S4 = a.summ + row_of(J, x);
    const int kq = J.kp >> 2, k = J.k;
    int acc = 0;
    for (int q = l; q < kq; q += gs) {
        const int4 g = __ldg(G4 + q);
        const int i = 4 * q;
        unsigned long long key[4] = {0, 0, 0, 0}, h[4] = {0, 0, 0, 0};
        ulonglong2 ev[4];
        bool on[4];
        on[0] = probe_start(table, mask, x, g.x, __ldg(S4 + 4 * q), i < k, sx, key[0], h[0], ev[0]);
        on[1] = probe_start(table, mask, x, g.y, __ldg(S4 + 4 * q + 1), i + 1 < k, sx, key[1], h[1], ev[1]);
        on[2] = probe_start(table, mask, x, g.z, __ldg(S4 + 4 * q + 2), i + 2 < k, sx, key[2], h[2], ev[2]);
        on[3] = probe_start(table, mask, x, g.w, __ldg(S4 + 4 * q + 3), i + 3 < k, sx, key[3], h[3], ev[3]);
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if (on[b]) acc += resolve(table, mask, key[b], h[b], ev[b]);
    }
    return acc;
}

// Partitions in which u and v carry the same label, plus the padding entries
// of this lane's quads: the two label rows (kq quads each) compared as int4.
__device__ __forceinline__ int row_part(const int* gu_row, const int* gv_row, int kq, int l, int gs)
{
    const int4* gu = reinterpret_cast<const int4*>(gu_row);
    const int4* gw = reinterpret_cast<const int4*>(gv_row);
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

// Automatic lanes per scored item (vertex, candidate or proposal): about ten
// partitions per lane for the largest k of the context.  Fewer lanes per item
// means more items per warp and fewer group reductions; timed on GB300 over
// 1..32 lanes, this was fastest for k = 20 (2 lanes) and k = 50 (8 lanes).
__host__ __device__ __forceinline__ int lanes_per_item(int k)
{
    int gs = 1;
    while (gs < 32 && gs * 10 < k) gs <<= 1;
    return gs;
}

// A_a for the vertices of running jobs whose cluster changed in the previous
// sweep (all of them in a run's first sweep): k for a singleton, else the
// summary part of its own cluster plus probes of the open partitions.  One
// group of lanes per vertex.
// ---- active set ------------------------------------------------------
// With cc_options.active_set, every move stamps its two clusters with the
// sweep's number, and a sweep after the first of a run re-scores only what
// the previous sweep can have changed.  v's gain towards a candidate x
// depends on A_a and |a| of its own cluster a and on |x| and A_x of x; v's
// candidates are the clusters of its neighbours, and a neighbour that moves
// stamps both its clusters.  So:
//   * A_a (aown[v]) is recomputed only if a was stamped;
//   * if neither a nor the target of v's previous bid was stamped, the
//     candidates that were not stamped keep their gains, and v's new bid is
//     the least of its previous bid and the bids of its stamped candidates:
//     only those are scored;
//   * otherwise (act[v] = 1) every candidate of v is scored.
// The first sweep of a run scores everything.

// kSingle: the context holds one job, so every vertex belongs to job 0 and
// the job is running whenever the sweep is not skipped.// kSingle: the context holds one job, so every vertex belongs to job 0 and
// the job is running whenever the sweep is not skipped.
template <bool kSingle>
__global__ void __launch_bounds__(kBlock, 4) k_own(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip) return;
    const unsigned long long mask = st->mask;
    const int gs = a.gs;
    const int lane = threadIdx.x & 31, l = lane & (gs - 1);
    const long long groups = (long long)gridDim.x * blockDim.x / gs;
    const JobInfo J0 = a.job[0];
    const int all = st->all_active, last = st->stamp - 1;
    // colour_batched: only the vertices of the current class, listed in vlist
    long long count = a.n, vbase = 0;
    if (a.colour_mode) {
        vbase = a.voff[st->cls];
        count = a.voff[st->cls + 1] - vbase;
    }
    for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x - lane) / gs; base < count;
         base += groups) {
        const long long idx = base + lane / gs;
        const bool valid = idx < count;
        const long long v = a.colour_mode ? (valid ? (long long)__ldg(a.vlist + vbase + idx) : 0) : idx;
        const int j = (kSingle || !valid) ? 0 : __ldg(a.jid + v);
        const bool run = valid && (kSingle || !a.js[j].stop);
        const int cv = run ? __ldg(a.C + v) : 0;
        // A_a is a function of v's cluster alone: it is recomputed only when
        // a vertex moved into or out of that cluster in the previous sweep
        // (or in a run's first sweep), and kept in aown[] otherwise; a colour
        // class was last scored several bodies ago, so it always recomputes
        const bool own = run && (a.colour_mode || all || a.chg[cv] == last);
        const bool on = own;
        if (a.active_set && run && l == 0) {
            // active set: every candidate again if a or the previous bid's
            // target changed
            const unsigned long long p = a.prev[v];
            const bool full = own || (p != kEmpty && a.chg[(int)(unsigned)(p & 0xffffffffull)] == last);
            a.act[v] = full ? 1 : 0;
        }
        // move-to-empty variant: the empty cluster with id v is a candidate
        // while no vertex carries that id (sizes are those of the sweep start)
        const bool iso = a.empty_moves && run && __ldg(a.size + v) == 0;
        if (!__any_sync(kFull, on || iso)) continue;  // nothing to score in this group of the warp
        const JobInfo J = kSingle ? J0 : a.job[j];
        const int sa = on ? __ldg(a.size + cv) : 1;
        const int* gv = a.G + row_of(J, on ? v : J.vo);
        int ex = 0, ub = 0, pb = 0;
        if (sa > 1) {
            summary_part(a, J, gv, cv, sa, l, gs, ex, ub);
            pb = probe_part(a, J, a.table, mask, gv, cv, sa, l, gs);
        }
        const int A = group_sum(ex + pb, gs);
        const int Aa = sa > 1 ? A : J.k;
        if (on && l == 0) a.aown[v] = Aa;
        if (iso && l == 0) {
            // Eq. objective3 with an empty target: 2 (A_a - k) - k (|a| - 1);
            // A_a is kept in aown[] when v's cluster did not change
            const int s_own = __ldg(a.size + cv);
            const int A_own = on ? Aa : a.aown[v];
            const int dD = 2 * (A_own - J.k) - J.k * (s_own - 1);
            if (dD < 0) atomicMin(&a.best[v], pack_key(dD, (int)v));
        }
    }
}

// Kept CSR entries of one warp, compacted in shared memory: up to kChunks
// chunks of 32 entries are gathered before scoring, so that the scoring
// rounds (32 / gs candidates each) run nearly full.
constexpr int kChunks = 4;
constexpr int kBoundSlots = 64;  // vertices of a window with a per-vertex bound (ids vbase .. vbase + 63)
struct EdgeScratch {
    int v[32 * kChunks], u[32 * kChunks], x[32 * kChunks], sx[32 * kChunks], sa[32 * kChunks], Aa[32 * kChunks],
        j[32 * kChunks];
    unsigned long long ubest[kBoundSlots];
    unsigned char open[32 * kChunks];
};

// CSR entries 32 at a time per warp: each lane reads one entry (v, u) and
// keeps it if v's job runs and u lies in another cluster than v (self-loops
// and repeats of the same (v, C[u]) inside the 32 entries are dropped, and so
// is a candidate whose gain is >= 0 even with A_x at its bound k |x|); the
// entries kept from kChunks chunks are then scored by groups of lanes.  A
// singleton {u} is scored from the two label rows; another cluster from its
// summary rows, then from probes of the open partitions, unless the lower
// bound on dD from the summary already rules the move out: a bound >= 0 (the
// move is never proposed), or a packed (bound, C[u]) not below an upper
// bound on v's final bid (v's least bid so far, or the summary's upper bound
// on another of v's candidates).  A move with dD < 0 bids its packed
// (dD, C[u]) at best[v] with an atomic minimum (a candidate kept in two
// chunks bids the same key twice).  The bids, and so the proposals, do not
// depend on which candidates the bounds skipped.  All group reductions are outside the branches, so every
// lane of the warp takes part in every shuffle.
template <bool kSingle>
__global__ void __launch_bounds__(kBlock, 4) k_edges(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip) return;
    __shared__ EdgeScratch sh[kWarpsPerBlock];
    const unsigned long long mask = st->mask;
    const int gs = a.gs, per = 32 / gs;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, l = lane & (gs - 1);
    const unsigned lt = (1u << lane) - 1u;
    EdgeScratch& es = sh[w];
    const JobInfo J0 = a.job[0];
    const int all = st->all_active, last = st->stamp - 1;
    const long long nwarps = (long long)gridDim.x * kWarpsPerBlock;
    constexpr long long span = 32 * kChunks;
    // colour_batched: only the CSR entries of the current class's vertices,
    // listed in eidx
    long long count = a.nnz, ebase = 0;
    if (a.colour_mode) {
        ebase = a.eoff[st->cls];
        count = a.eoff[st->cls + 1] - ebase;
    }
    for (long long base = ((long long)blockIdx.x * kWarpsPerBlock + w) * span; base < count; base += nwarps * span) {
        // singleton candidates fill the scratch from the front, the others
        // from the back, so that scoring rounds take one path each
        int ns = 0, nt = 0;
        // the loads of all kChunks chunks first (entries, then clusters), so
        // that their latencies overlap; then each chunk's votes and compaction
        int vc[kChunks], uc[kChunks], xc[kChunks], cvc[kChunks], jc[kChunks];
#pragma unroll
        for (int c = 0; c < kChunks; ++c) {
            const long long ep = base + c * 32 + lane;
            vc[c] = 0;
            uc[c] = 0;
            jc[c] = 0;
            if (ep < count) {
                const long long e = a.colour_mode ? (long long)__ldg(a.eidx + ebase + ep) : ep;
                vc[c] = __ldg(a.src + e);
                uc[c] = __ldg(a.col + e);
                if (!kSingle) jc[c] = __ldg(a.jid + vc[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < kChunks; ++c) {
            const long long ep = base + c * 32 + lane;
            xc[c] = -1;
            cvc[c] = 0;
            if (ep < count && uc[c] != vc[c] && (kSingle || !a.js[jc[c]].stop)) {
                xc[c] = __ldg(a.C + uc[c]);
                cvc[c] = __ldg(a.C + vc[c]);
            }
        }
        for (int c = 0; c < kChunks; ++c) {
            const long long ep = base + c * 32 + lane;
            const int v = vc[c], u = uc[c], j = jc[c];
            int x = xc[c];
            const int cv = cvc[c];
            // entries of stopped jobs are not scored; a chunk of only such
            // entries is skipped whole
            const bool live = ep < count && (kSingle || !a.js[j].stop);
            if (__all_sync(kFull, !live)) continue;
            if (live && x >= 0) {
                if (x == cv) x = -1;
                // active set: only candidates that changed, unless v is
                // scored in full
                else if (a.active_set && !all && !a.act[v] && a.chg[x] != last) x = -1;
            }
            const unsigned long long pair = x >= 0 ? ((unsigned long long)(unsigned)v << 32) | (unsigned)x : kEmpty;
            const unsigned same = __match_any_sync(kFull, pair);
            bool keep = x >= 0 && (__ffs(same) - 1) == lane;
            int sx = 0, sa = 0, Aa = 0;
            if (keep) {
                sx = __ldg(a.size + x);
                sa = __ldg(a.size + cv);
                Aa = __ldg(a.aown + v);
                // exact prune: n(x, i, l) <= |x| gives A_x <= k |x|, so a move
                // whose gain is >= 0 even at that bound is never proposed
                const long long k = kSingle ? J0.k : a.job[j].k;
                if (2 * ((long long)Aa - k - k * sx) - k * ((long long)sa - 1 - sx) >= 0) keep = false;
            }
            const bool sgl = keep && sx == 1;
            const unsigned ks = __ballot_sync(kFull, sgl), kt = __ballot_sync(kFull, keep && !sgl);
            if (keep) {
                const int p = sgl ? ns + __popc(ks & lt) : (int)span - 1 - (nt + __popc(kt & lt));
                es.v[p] = v;
                es.u[p] = u;
                es.x[p] = x;
                if (!kSingle) es.j[p] = j;
                es.sx[p] = sx;
                es.sa[p] = sa;
                es.Aa[p] = Aa;
            }
            ns += __popc(ks);
            nt += __popc(kt);
        }
        __syncwarp();
        // singleton candidates: two label rows compared, half the lanes per
        // item of the cluster candidates (a plain streaming compare)
        {
            const int gr = gs > 1 ? gs >> 1 : 1, pr = 32 / gr, lr = lane & (gr - 1);
            for (int r0 = 0; r0 < ns; r0 += pr) {
                const int q = r0 + lane / gr;
                const bool valid = q < ns;
                const int ev = valid ? es.v[q] : 0, eu = valid ? es.u[q] : 0, ex_ = valid ? es.x[q] : 0;
                const int sa = valid ? es.sa[q] : 0, Aa = valid ? es.Aa[q] : 0;
                const JobInfo J = kSingle ? J0 : a.job[valid ? es.j[q] : 0];
                int part = 0;
                if (valid) part = row_part(a.G + row_of(J, eu), a.G + row_of(J, ev), J.kp >> 2, lr, gr);
                part = group_sum(part, gr);
                if (valid && lr == 0) {
                    const int k = J.k, A = part - (J.kp - k);
                    const int dD = 2 * (Aa - k - A) - k * (sa - 1 - 1);
                    if (dD < 0) atomicMin(&a.best[ev], pack_key(dD, ex_));
                }
            }
        }
        // other clusters, in two passes.  Pass 1: the summary rows give each
        // candidate an exact part and an upper bound ub on A_x, so a least
        // dD (lo, with A = ub) and a largest one (hi, with A = part); one
        // that the summary settles (ub == part) bids at once.  The least
        // packed (hi, x) with hi < 0 over a vertex's candidates of the window
        // bounds that vertex's final bid from above.  Pass 2: the candidates
        // whose packed (lo, x) lies below that bound and below the vertex's
        // least bid so far are listed, and probed in full rounds of gs lanes
        // each; the others cannot be the vertex's least bid.
        for (int t = lane; t < kBoundSlots; t += 32) es.ubest[t] = kEmpty;
        const int vbase = nt > 0 ? es.v[span - 1] : 0;
        __syncwarp();
        for (int r0 = 0; r0 < nt; r0 += per) {
            const int qq = r0 + lane / gs;
            const bool valid = qq < nt;
            const int q = (int)span - 1 - qq;
            const int ev = valid ? es.v[q] : 0, ex_ = valid ? es.x[q] : 0;
            const int sx = valid ? es.sx[q] : 0, sa = valid ? es.sa[q] : 0, Aa = valid ? es.Aa[q] : 0;
            const JobInfo J = kSingle ? J0 : a.job[valid ? es.j[q] : 0];
            const int k = J.k;
            const int* gv = a.G + row_of(J, valid ? ev : J.vo);
            int part = 0, ub = 0;
            if (valid) summary_part(a, J, gv, ex_, sx, l, gs, part, ub);
            part = group_sum(part, gs);
            ub = group_sum(ub, gs);
            if (valid && l == 0) {
                const int base = 2 * (Aa - k) - k * (sa - 1 - sx);  // dD = base - 2 A
                const int lo = base - 2 * ub, hi = base - 2 * part;
                const unsigned d = (unsigned)(ev - vbase);
                if (hi < 0 && d < (unsigned)kBoundSlots) atomicMin(&es.ubest[d], pack_key(hi, ex_));
                if (ub == part) {
                    if (lo < 0) atomicMin(&a.best[ev], pack_key(lo, ex_));
                    es.u[q] = 0;  // settled
                } else {
                    es.u[q] = lo;
                    es.sa[q] = base;
                    es.Aa[q] = part;
                }
            }
        }
        __syncwarp();
        int no = 0;
        for (int c0 = 0; c0 < nt; c0 += 32) {
            const int qq = c0 + lane;
            const int q = (int)span - 1 - qq;
            bool open = false;
            if (qq < nt) {
                const int lo = es.u[q];
                if (lo < 0) {
                    const int ev = es.v[q];
                    const unsigned d = (unsigned)(ev - vbase);
                    unsigned long long thr = __ldcg(a.best + ev);
                    if (d < (unsigned)kBoundSlots && es.ubest[d] < thr) thr = es.ubest[d];
                    open = pack_key(lo, es.x[q]) < thr;
                }
            }
            const unsigned bal = __ballot_sync(kFull, open);
            if (open) es.open[no + __popc(bal & lt)] = (unsigned char)q;
            no += __popc(bal);
        }
        __syncwarp();
        for (int r0 = 0; r0 < no; r0 += per) {
            const int qi = r0 + lane / gs;
            const bool valid = qi < no;
            const int q = valid ? (int)es.open[qi] : 0;
            const int ev = valid ? es.v[q] : 0, ex_ = valid ? es.x[q] : 0, sx = valid ? es.sx[q] : 0;
            const JobInfo J = kSingle ? J0 : a.job[valid ? es.j[q] : 0];
            const int* gv = a.G + row_of(J, valid ? ev : J.vo);
            int pb = 0;
            if (valid) pb = probe_part(a, J, a.table, mask, gv, ex_, sx, l, gs);
            pb = group_sum(pb, gs);
            if (valid && l == 0) {
                const int dD = es.sa[q] - 2 * (es.Aa[q] + pb);
                if (dD < 0) atomicMin(&a.best[ev], pack_key(dD, ex_));
            }
        }
        __syncwarp();
    }
}

// Turns the bids into the proposal list (v, a, b, dD), counts them per job and
// clears best[].  Each block gathers its proposals in shared memory and
// appends them with one global atomic.
__global__ void __launch_bounds__(kBlock) k_collect(SweepArgs a)
{
    extern __shared__ long long dyn_jobs[];
    DevState* st = a.st;
    if (st->skip) return;
    __shared__ int4 sbuf[kBlock];
    __shared__ int s_cnt, s_keys;
    __shared__ unsigned long long s_base;
    JobAcc acc(job_smem_init(a.jobs, dyn_jobs), reinterpret_cast<long long*>(&a.js[0].nprop), kJobStride);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long b0 = (long long)blockIdx.x * blockDim.x; b0 < a.n; b0 += stride) {
        if (threadIdx.x == 0) {
            s_cnt = 0;
            s_keys = 0;
        }
        __syncthreads();
        const long long v = b0 + threadIdx.x;
        if (v < a.n) {
            unsigned long long key = a.best[v];
            if (key != kEmpty) a.best[v] = kEmpty;
            if (a.active_set) {
                // a vertex scored only on its changed candidates keeps its
                // previous bid if that is still the least; a vertex of a
                // stopped job bids nothing
                if (a.js[a.jid[v]].stop) key = kEmpty;
                else if (!st->all_active && !a.act[v] && a.prev[v] < key) key = a.prev[v];
                a.prev[v] = key;
            }
            if (key != kEmpty) {
                const int job = a.jid[v];
                acc.add(job, 1);
                const int p = atomicAdd(&s_cnt, 1);
                atomicAdd(&s_keys, a.job[job].k);
                sbuf[p] = make_int4((int)v, a.C[v], (int)(unsigned)(key & 0xffffffffull), key_gain(key));
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && s_cnt > 0) {
            s_base = atomicAdd(&st->nprop, (unsigned long long)s_cnt);
            atomicAdd(&st->pkeys, (unsigned long long)s_keys);
        }
        __syncthreads();
        for (int p = threadIdx.x; p < s_cnt; p += blockDim.x) {
            const int4 q = sbuf[p];
            const unsigned long long jj = s_base + p;
            a.pv[jj] = q.x;
            a.pa[jj] = q.y;
            a.pb[jj] = q.z;
            a.pg[jj] = q.w;
        }
        __syncthreads();
    }
    job_acc_finish(acc, a.jobs);
}

// ---- heavy sweeps --------------------------------------------------------
// When the proposals move a large share of the label rows (more than 1/8 of
// sum_j k_j n_j; for one job |P| > n / 8), or always with sweep_mode 2, never
// with sweep_mode 1, or when the table does not hold the
// counts of C yet (the singleton start), dF(P1) is taken from a rebuild
// instead of from staged deltas: P1 is applied to C in place (the movers' old
// clusters stay in the proposal list), the table and its summary rows are
// rebuilt from the new C, and F' - F is dF(P1) exactly for every job.  A job
// whose dF is negative has committed P1 (mode 3); any other job's moves are
// undone, the table is rebuilt from C again and its matching fallback runs as
// in a light sweep (mode 2).

__global__ void k_route(SweepArgs a)
{
    const unsigned long long total_keys = a.keys;
    DevState* st = a.st;
    st->heavy = 0;
    if (st->skip || st->err || st->nprop == 0) return;
    // light when the proposals move at most 1/8 of all label rows (for one
    // job: |P| <= n / 8)
    const bool light = a.sweep_mode == 1 || (a.sweep_mode == 0 && st->pkeys * 8 <= total_keys);
    if (st->tvalid && light) return;
    st->heavy = 1;
    // keys after applying P1: every vertex gives at most k, every mover at most k new ones
    unsigned long long bound = (st->tvalid ? (unsigned long long)st->live : total_keys) +
                               st->pkeys;
    if (bound > total_keys) bound = total_keys;
    unsigned long long c = a.cap_min;
    while (c < 2 * bound && c < a.mask_max + 1) c <<= 1;
    // First a tight capacity: the occupied slots of the sweep start (the
    // moves of a heavy sweep mostly merge keys) at load <= 1/2, with room
    // below the fill limit for the new keys of a following light sweep
    // (2 x sum k n / 8 at most).  The rebuild checks that the keys fit
    // (k_build_check) and otherwise builds again at c.
    const unsigned long long est = st->tvalid ? st->used : total_keys;
    const unsigned long long room = 2 * ((total_keys + 7) / 8);
    unsigned long long t = a.cap_min;
    while ((t < 2 * est || t - (t >> 3) < est + room) && t < c) t <<= 1;
    st->safe_mask = c - 1;
    st->tight = (t < c && a.tight_mode != 1) ? 1 : 0;
    if (!st->tight) t = c;
    st->new_mask = t - 1;
    st->rebuild = 1;
}

// Singleton guard on every proposal (sizes of the sweep start); counts |P1| per job.
__global__ void k_h_mark(SweepArgs a)
{
    extern __shared__ long long dyn_jobs[];
    DevState* st = a.st;
    if (st->skip || !st->heavy) return;
    JobAcc acc(job_smem_init(a.jobs, dyn_jobs), reinterpret_cast<long long*>(&a.js[0].np1), kJobStride);
    const long long np = (long long)st->nprop;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += stride) {
        const int ca = a.pa[p], cb = a.pb[p];
        const bool keep = !(a.size[ca] == 1 && a.size[cb] == 1) || cb < ca;
        a.pflag[p] = keep ? 1 : 0;
        if (keep) acc.add(a.jid[a.pv[p]], 1);
    }
    job_acc_finish(acc, a.jobs);
}

// Applies (undo = 0) or undoes (undo = 1, jobs that roll back only) the kept
// proposals on C and the sizes.
__global__ void k_h_apply(SweepArgs a, int undo)
{
    DevState* st = a.st;
    if (st->skip || !st->heavy || (undo && !st->rollback)) return;
    const long long np = (long long)st->nprop;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += stride) {
        if (!a.pflag[p]) continue;
        const int v = a.pv[p];
        if (undo && !a.js[a.jid[v]].rollback) continue;
        const int ca = a.pa[p], cb = a.pb[p];
        a.C[v] = undo ? ca : cb;
        atomicAdd(&a.size[ca], undo ? 1 : -1);
        atomicAdd(&a.size[cb], undo ? -1 : 1);
        if (!undo) {
            a.chg[ca] = st->stamp;
            a.chg[cb] = st->stamp;
        }
    }
}

// The size part of F' per job (k sum_c s_c^2); the table part was added by the
// summary pass of the rebuild.
__global__ void k_h_eval(SweepArgs a)
{
    extern __shared__ long long dyn_jobs[];
    DevState* st = a.st;
    if (st->skip || !st->heavy || st->err) return;
    JobAcc acc(job_smem_init(a.jobs, dyn_jobs), &a.js[0].recompute, kJobStride);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < a.n; c += stride) {
        const long long sz = a.size[c];
        if (sz > 0) {
            const int job = a.jid[c];
            acc.add(job, (long long)a.job[job].k * sz * sz);
        }
    }
    job_acc_finish(acc, a.jobs);
}

__global__ void k_h_decide(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip || !st->heavy) return;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < a.jobs; j += gridDim.x * blockDim.x) {
        JobState& s = a.js[j];
        if (s.stop) continue;
        if (st->err) {
            s.mode = 0;
            continue;
        }
        const long long dF = s.recompute + s.partition_sq - s.F;
        s.dF_p1 = s.np1 > 0 ? dF : 0;
        if (s.np1 > 0 && dF < 0) {
            s.mode = 3;
            s.dF = dF;
            s.moves = s.np1;
        } else {
            s.mode = s.nprop > 0 ? 2 : 0;
            s.dF = 0;
            s.moves = 0;
            if (s.np1 > 0) s.rollback = 1;
            // the rollback rebuilds at the capacity that holds every key the
            // sweep can create, so that the matching fallback's inserts fit;
            // a job that falls back without moves to undo also needs that
            // room when the heavy rebuild was a tight one
            if (s.np1 > 0 || (s.mode == 2 && st->mask != st->safe_mask)) {
                st->rollback = 1;
                st->rebuild = 1;
                st->new_mask = st->safe_mask;
            }
        }
    }
}

// ---- light sweeps -------------------------------------------------------

// Occupancy above which a sweep is abandoned and retried in a larger table.
__device__ __forceinline__ unsigned long long fill_limit(unsigned long long mask)
{
    return (mask + 1) - ((mask + 1) >> 3);
}

// Adds the warp's new slots to st->used and flags an overflow past the limit.
// All lanes must call it.
__device__ __forceinline__ void count_inserts(DevState* st, int mine, unsigned long long mask)
{
    int x = mine;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    if ((threadIdx.x & 31) == 0 && x > 0) {
        const unsigned long long old = atomicAdd(&st->used, (unsigned long long)x);
        if (old + x > fill_limit(mask)) st->overflow = 1;
    }
}

// The light-path kernels give each proposal a group of gs lanes: the lanes
// split the job's partitions, and the group's first lane does the per-proposal
// work (flags, sizes, bids, sums).  Items of one warp: 32 / gs proposals.
#define PROPOSAL_LOOP(np)                                                                                  \
    const int gs = a.gs, per = 32 / gs;                                                                   \
    const int lane = threadIdx.x & 31, l = lane & (gs - 1);                                               \
    const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;                      \
    const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;                                     \
    for (long long b0 = warp0 * per; b0 < (np); b0 += nwarp * per)

__device__ __forceinline__ long long group_sum64(long long x, int gs)
{
    for (int o = gs >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

// Singleton guard, and staged deltas of the kept proposals.  Staging never
// fails: if the table runs short of slots the sweep is abandoned
// (st->overflow) before anything is committed, and the sweep end schedules a
// larger table and a retry.
__global__ void k_stage(SweepArgs a)
{
    extern __shared__ long long dyn_jobs[];
    DevState* st = a.st;
    if (st->skip || st->err || st->heavy) return;
    JobAcc acc(job_smem_init(a.jobs, dyn_jobs), reinterpret_cast<long long*>(&a.js[0].np1), kJobStride);
    const unsigned long long mask = st->mask;
    const long long np = (long long)st->nprop;
    PROPOSAL_LOOP(np)
    {
        const long long p = b0 + lane / gs;
        int job = -1, ins_count = 0;
        if (p < np) {
            const int v = a.pv[p], ca = a.pa[p], cb = a.pb[p];
            const bool keep = !(a.size[ca] == 1 && a.size[cb] == 1) || cb < ca;
            if (l == 0) a.pflag[p] = keep ? 1 : 0;
            if (keep) {
                const int j = a.jid[v];
                const JobInfo& J = a.job[j];
                if (l == 0) {
                    job = j;
                    atomicAdd(&a.dsize[ca], -1);
                    atomicAdd(&a.dsize[cb], 1);
                }
                const int* gv = a.G + row_of(J, v);
                for (int i = l; i < J.k; i += gs) {
                    const int g = gv[i];
                    bool ins = false;
                    const long long sa = table_find(a.table, mask, ckey(ca, g));
                    const long long sb = table_find_or_insert(a.table, mask, ckey(cb, g), &ins);
                    ins_count += ins;
                    if (sa < 0) {
                        set_err(st, CC_ERR_INVALID);  // the vertex's own key must exist
                    } else if (sb < 0) {
                        st->overflow = 1;
                    } else {
                        atomicAdd(&a.table[sa].dlt, -1);
                        atomicAdd(&a.table[sb].dlt, 1);
                    }
                }
            }
        }
        count_inserts(st, ins_count, mask);
        if (job >= 0) acc.add(job, 1);
    }
    job_acc_finish(acc, a.jobs);
}

// dF(P1) per job = k sum_c ((s+ds)^2 - s^2) - 2 sum_keys ((n+dn)^2 - n^2),
// written as a sum over the staged contributions: each +-1 added to an entry
// x with final delta d_x contributes +-(2 x + d_x).
__global__ void k_eval(SweepArgs a)
{
    extern __shared__ long long dyn_jobs[];
    DevState* st = a.st;
    if (st->skip || st->err || st->overflow || st->heavy) return;
    JobAcc acc(job_smem_init(a.jobs, dyn_jobs), &a.js[0].dF, kJobStride);
    const unsigned long long mask = st->mask;
    const long long np = (long long)st->nprop;
    PROPOSAL_LOOP(np)
    {
        const long long p = b0 + lane / gs;
        long long keys = 0, sizes = 0;
        int job = -1;
        if (p < np && a.pflag[p]) {
            const int v = a.pv[p], ca = a.pa[p], cb = a.pb[p];
            const int j = a.jid[v];
            const JobInfo& J = a.job[j];
            const int* gv = a.G + row_of(J, v);
            for (int i = l; i < J.k; i += gs) {
                const int g = gv[i];
                const long long sa = table_find(a.table, mask, ckey(ca, g));
                const long long sb = table_find(a.table, mask, ckey(cb, g));
                if (sa < 0 || sb < 0) {
                    set_err(st, CC_ERR_INVALID);  // staged keys must exist
                    continue;
                }
                const Slot* A = a.table + sa;
                const Slot* B = a.table + sb;
                keys += -(2LL * A->cnt + A->dlt) + (2LL * B->cnt + B->dlt);
            }
            if (l == 0) {
                job = j;
                sizes = (long long)J.k * (-(2LL * a.size[ca] + a.dsize[ca]) + (2LL * a.size[cb] + a.dsize[cb]));
            }
        }
        keys = group_sum64(keys, gs);
        if (job >= 0) acc.add(job, -2 * keys + sizes);
    }
    job_acc_finish(acc, a.jobs);
}

__global__ void k_decide(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip || st->heavy) return;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < a.jobs; j += gridDim.x * blockDim.x) {
        JobState& s = a.js[j];
        if (s.stop) continue;
        if (st->err || st->overflow) {
            s.mode = 0;
            continue;
        }
        if (s.np1 > 0 && s.dF < 0) {
            s.mode = 1;
            s.dF_p1 = s.dF;
            s.moves = s.np1;
        } else if (s.nprop > 0) {
            s.mode = 2;
            s.dF_p1 = s.np1 > 0 ? s.dF : 0;
            s.dF = 0;
            s.moves = 0;
        } else {
            s.mode = 0;
            s.dF = 0;
        }
    }
}

// Proposals of a job that falls back to the matching (mode 2): undo their
// staged deltas (light sweeps) and bid (dD, v) at both clusters.
__global__ void k_bid(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip || st->err) return;
    const bool staged = !st->heavy;
    const unsigned long long mask = st->mask;
    const long long np = (long long)st->nprop;
    PROPOSAL_LOOP(np)
    {
        const long long p = b0 + lane / gs;
        if (p >= np) continue;
        const int v = a.pv[p], ca = a.pa[p], cb = a.pb[p];
        const int j = a.jid[v];
        if (a.js[j].mode != 2) continue;
        if (staged && a.pflag[p]) {
            const JobInfo& J = a.job[j];
            const int* gv = a.G + row_of(J, v);
            for (int i = l; i < J.k; i += gs) {
                const int g = gv[i];
                const long long sa = table_find(a.table, mask, ckey(ca, g));
                const long long sb = table_find(a.table, mask, ckey(cb, g));
                if (sa >= 0) a.table[sa].dlt = 0;
                if (sb >= 0) a.table[sb].dlt = 0;
            }
            if (l == 0) {
                a.dsize[ca] = 0;
                a.dsize[cb] = 0;
            }
        }
        if (l == 0) {
            const unsigned long long key = pack_key(a.pg[p], v);
            atomicMin(&a.best[ca], key);
            atomicMin(&a.best[cb], key);
        }
    }
}

// Fallback: a proposal is committed iff its (dD, v) is the least at both of
// its clusters; the committed moves touch pairwise-disjoint clusters, so
// their objective changes add exactly.  This pass marks the winners and
// inserts their target keys.  It runs before any count of any job changes,
// so that a table overflow abandons the whole sweep with nothing committed.
__global__ void k_match_keys(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip || st->err) return;
    const unsigned long long mask = st->mask;
    const long long np = (long long)st->nprop;
    PROPOSAL_LOOP(np)
    {
        const long long p = b0 + lane / gs;
        int ins_count = 0;
        if (p < np) {
            const int v = a.pv[p], ca = a.pa[p], cb = a.pb[p];
            const int j = a.jid[v];
            const unsigned long long key = pack_key(a.pg[p], v);
            if (a.js[j].mode == 2 && a.best[ca] == key && a.best[cb] == key) {
                if (l == 0) a.pflag[p] = 2;
                const JobInfo& J = a.job[j];
                const int* gv = a.G + row_of(J, v);
                for (int i = l; i < J.k; i += gs) {
                    bool ins = false;
                    if (table_find_or_insert(a.table, mask, ckey(cb, gv[i]), &ins) < 0) st->overflow = 1;
                    ins_count += ins;
                }
            }
        }
        count_inserts(st, ins_count, mask);
    }
}

// The light commit of P1 (mode 1: C, the staged size and count deltas folded
// in) or the move of a matching winner (mode 2).  Skipped entirely after an
// overflow.
__global__ void k_commit(SweepArgs a)
{
    extern __shared__ long long dyn_jobs[];
    DevState* st = a.st;
    if (st->skip || st->err || st->overflow) return;
    long long* sh = job_smem_init(2 * a.jobs <= kSmemJobs ? a.jobs : 0, dyn_jobs);
    if (sh) {
        for (int j = threadIdx.x; j < a.jobs; j += blockDim.x) sh[a.jobs + j] = 0;
        __syncthreads();
    }
    JobAcc mv(sh, reinterpret_cast<long long*>(&a.js[0].moves), kJobStride);
    JobAcc df(sh ? sh + a.jobs : nullptr, &a.js[0].dF, kJobStride);
    const unsigned long long mask = st->mask;
    const long long np = (long long)st->nprop;
    PROPOSAL_LOOP(np)
    {
        const long long p = b0 + lane / gs;
        long long live = 0, dF = 0, moved = 0;
        int job = -1;
        if (p < np) {
            const int v = a.pv[p], ca = a.pa[p], cb = a.pb[p];
            const int j = a.jid[v];
            const int mode = a.js[j].mode;
            const JobInfo& J = a.job[j];
            const int* gv = a.G + row_of(J, v);
            if (mode == 1 && a.pflag[p]) {
                if (l == 0) {
                    a.C[v] = cb;
                    a.chg[ca] = st->stamp;
                    a.chg[cb] = st->stamp;
                    int d = atomicExch(&a.dsize[ca], 0);
                    if (d) atomicAdd(&a.size[ca], d);
                    d = atomicExch(&a.dsize[cb], 0);
                    if (d) atomicAdd(&a.size[cb], d);
                }
                for (int i = l; i < J.k; i += gs) {
                    const int g = gv[i];
#pragma unroll
                    for (int side = 0; side < 2; ++side) {
                        const long long si = table_find(a.table, mask, ckey(side ? cb : ca, g));
                        if (si < 0) {
                            set_err(st, CC_ERR_INVALID);
                            continue;
                        }
                        Slot* s = a.table + si;
                        const int dd = atomicExch(&s->dlt, 0);
                        if (dd) {
                            const int old = atomicAdd(&s->cnt, dd);
                            live += (old == 0) - (old + dd == 0);
                            summ_update(a, s->key, dd);
                        }
                    }
                }
            } else if (mode == 2 && a.pflag[p] == 2) {
                if (l == 0) {
                    job = j;
                    a.C[v] = cb;
                    a.chg[ca] = st->stamp;
                    a.chg[cb] = st->stamp;
                    atomicAdd(&a.size[ca], -1);
                    atomicAdd(&a.size[cb], 1);
                    moved = 1;
                    dF = 2LL * a.pg[p];
                }
                for (int i = l; i < J.k; i += gs) {
                    const int g = gv[i];
                    const long long sa = table_find(a.table, mask, ckey(ca, g));
                    const long long sb = table_find(a.table, mask, ckey(cb, g));
                    if (sa < 0 || sb < 0) {
                        set_err(st, CC_ERR_INVALID);
                        continue;
                    }
                    const int oa = atomicAdd(&a.table[sa].cnt, -1);
                    const int ob = atomicAdd(&a.table[sb].cnt, 1);
                    live += (ob == 0) - (oa == 1);
                    summ_update(a, ckey(ca, g), -1);
                    summ_update(a, ckey(cb, g), 1);
                }
            }
        }
        warp_add64(live, &st->live);
        if (job >= 0) {
            mv.add(job, moved);
            df.add(job, dF);
        }
    }
    job_acc_finish(mv, a.jobs);
    job_acc_finish(df, a.jobs);
}

__global__ void k_match_reset(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip) return;
    const long long np = (long long)st->nprop;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += stride) {
        if (a.js[a.jid[a.pv[p]]].mode != 2) continue;
        a.best[a.pa[p]] = kEmpty;
        a.best[a.pb[p]] = kEmpty;
    }
}

// Per job: objective, history record, stop.  An abandoned sweep changes no job.
__global__ void k_end_jobs(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip || st->err || st->overflow) return;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < a.jobs; j += gridDim.x * blockDim.x) {
        JobState& s = a.js[j];
        if (s.stop) continue;
        if (s.mode != 0) s.F += s.dF;
        cc_sweep_info r;
        r.proposals = (int64_t)s.nprop;
        r.p1 = (int64_t)s.np1;
        r.dF_p1 = s.dF_p1;
        r.fallback = s.mode == 2 ? 1 : 0;
        r.moves = (int64_t)s.moves;
        r.F = s.F;
        if (a.colour_mode) {
            // a colour class: add it to the sweep's totals; the sweep ends
            // with its last class
            s.t_prop += r.proposals;
            s.t_p1 += r.p1;
            s.t_dFp1 += r.dF_p1;
            s.t_fb += r.fallback;
            s.t_moves += r.moves;
            if (st->cls + 1 < st->ncls) continue;
            r.proposals = s.t_prop;
            r.p1 = s.t_p1;
            r.dF_p1 = s.t_dFp1;
            r.fallback = s.t_fb;
            r.moves = s.t_moves;
            s.t_prop = s.t_p1 = s.t_dFp1 = s.t_fb = s.t_moves = 0;
        }
        if (s.sweeps < a.hist_cap) a.hist[(long long)j * a.hist_cap + s.sweeps] = r;
        s.sweeps += 1;
        s.run_sweeps += 1;
        if (r.proposals == 0 || s.run_sweeps >= st->run_limit) s.stop = 1;
        else atomicAdd(&st->active, 1);
    }
}

__global__ void k_end(SweepArgs a)
{
    DevState* st = a.st;
    if (st->skip) return;
    st->run_bodies += 1;
    if (st->err) {
        st->stop = 1;
        return;
    }
    const unsigned long long cap = st->mask + 1;
    if (st->overflow) {
        // nothing was committed: retry this sweep after rebuilding into twice
        // the capacity (the staged deltas are discarded with the old table).
        // A heavy sweep sizes its table for every key it can create, so it
        // cannot overflow; if it did, jobs that kept P1 have moved already
        // and a retry would be wrong, so that is reported instead.
        if (cap >= a.mask_max + 1 || st->heavy) {
            set_err(st, CC_ERR_TABLE_FULL);
            st->stop = 1;
            return;
        }
        st->new_mask = 2 * cap - 1;
        st->abort = 1;
        st->rebuild = 1;
        st->retries += 1;
        st->stamp -= 1;  // the retry is the same sweep: it reuses the stamp
        return;
    }
    st->all_active = 0;
    if (a.colour_mode && st->cls + 1 < st->ncls) {
        st->cls += 1;  // the sweep goes on with the next colour class
        st->stop = 0;
    } else {
        st->cls = 0;
        st->stop = st->active == 0 ? 1 : 0;
    }
    // compaction: rebuild without the dead keys when occupied slots pass one
    // half of the capacity; the new capacity holds the live keys plus k x
    // (proposals of this sweep), a forecast of the next sweep's new keys, at
    // load <= 1/2.  (Summary rows settle most of each score, so a table larger
    // than needed costs little; it is not shrunk otherwise.)
    const unsigned long long live = (unsigned long long)st->live;
    const unsigned long long want = 2 * (live + st->pkeys);
    unsigned long long c = a.cap_min;
    while (c < want && c < a.mask_max + 1) c <<= 1;
    if (st->tvalid && st->used > cap / 2) {
        st->new_mask = c - 1;
        st->rebuild = 1;
    } else {
        st->rebuild = 0;
    }
}

// Regions of a sweep that run only when needed.  In a captured graph each is
// an IF node whose condition a one-thread gate kernel sets from the control
// block, so a sweep that does not need a region skips its launches instead of
// running kernels that return at once.
enum Gate { kGateHeavy = 0, kGateRollback = 1, kGateLight = 2, kGateRebuild = 3, kGateRetry = 4, kGateHeavyEval = 5 };

__global__ void k_gate(cudaGraphConditionalHandle h, DevState* st, int which, int kernels)
{
    const bool run = !st->skip && !st->err;
    bool on = false;
    if (which == kGateHeavy || which == kGateHeavyEval) on = run && st->heavy;
    else if (which == kGateRetry) on = run && st->heavy && st->rebuild;
    else if (which == kGateRollback) on = run && st->heavy && st->rollback;
    else if (which == kGateLight) on = run && !st->heavy && st->nprop > 0;
    else on = st->rebuild && !st->err;
    if (on) st->region_launches += (unsigned long long)kernels;
    cudaGraphSetConditional(h, on ? 1u : 0u);
}

// Opens an IF region in the graph being captured on s: the gate kernel, then
// the conditional node, whose body is captured on b until close_region.
cudaError_t open_region(cudaStream_t s, cudaStream_t b, DevState* st, Gate which, int kernels)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureUnsupported;
    cudaGraphConditionalHandle h = 0;
    e = cudaGraphConditionalHandleCreate(&h, g, 0, 0);
    if (e != cudaSuccess) return e;
    k_gate<<<1, 1, 0, s>>>(h, st, (int)which, kernels);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t nd = 0;
    e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edges, &nd);
    if (e != cudaSuccess) return e;
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    e = cudaGraphAddNode(&node, g, deps, edges, nd, &p);
    if (e != cudaSuccess) return e;
    e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) return e;
    return cudaStreamBeginCaptureToGraph(b, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal);
}

cudaError_t close_region(cudaStream_t b)
{
    cudaGraph_t g = nullptr;
    return cudaStreamEndCapture(b, &g);
}

// End of one body of a run loop: go on while the run has not stopped, has no
// error and has run fewer than `budget` sweep bodies.
__global__ void k_loop_gate(cudaGraphConditionalHandle h, DevState* st, int budget)
{
    const bool more = !st->stop && !st->err && st->run_bodies < budget;
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

inline int jobs_grid(int jobs)
{
    int g = (jobs + 255) / 256;
    return g < 1 ? 1 : g;
}

}  // namespace

int lanes_for_k(int k)
{
    return lanes_per_item(k);
}

__global__ void k_clear_bids(SweepArgs a)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += stride) a.best[v] = kEmpty;
}

cudaError_t launch_propose_probe(const SweepArgs& a, int grid, cudaStream_t s)
{
    if (a.jobs == 1) {
        k_own<true><<<grid, kBlock, 0, s>>>(a);
        k_edges<true><<<grid, kBlock, 0, s>>>(a);
    } else {
        k_own<false><<<grid, kBlock, 0, s>>>(a);
        k_edges<false><<<grid, kBlock, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_clear_bids(const SweepArgs& a, int grid, cudaStream_t s)
{
    k_clear_bids<<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t prepare_propose(int* blocks_per_sm)
{
    int single = 0, multi = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&single, k_edges<true>, kBlock, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&multi, k_edges<false>, kBlock, 0);
    *blocks_per_sm = single < multi ? single : multi;
    return e;
}

cudaError_t capture_run_loop(const SweepArgs& a, long long rows, int grid, cudaStream_t s, cudaStream_t loop,
                             cudaStream_t body, int budget)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edges, &nd);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureUnsupported;
    // the loop is entered once per launch (default value 1); each body's gate
    // decides whether another follows
    cudaGraphConditionalHandle h = 0;
    e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return e;
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    e = cudaGraphAddNode(&node, g, deps, edges, nd, &p);
    if (e != cudaSuccess) return e;
    e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCaptureToGraph(loop, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    e = launch_sweep(a, rows, grid, loop, nullptr, nullptr, body);
    if (e == cudaSuccess) {
        k_loop_gate<<<1, 1, 0, loop>>>(h, a.st, budget);
        e = cudaGetLastError();
    }
    cudaGraph_t lg = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(loop, &lg);
    return e != cudaSuccess ? e : e2;
}

cudaError_t launch_run_begin(const SweepArgs& a, int limit, cudaStream_t s)
{
    k_run_begin<<<jobs_grid(a.jobs), 256, 0, s>>>(a, limit);
    return cudaGetLastError();
}

cudaError_t launch_sweep(const SweepArgs& a, long long rows, int grid, cudaStream_t s, cudaEvent_t prop0,
                         cudaEvent_t prop1, cudaStream_t body)
{
    const int g2 = grid;
    const int jg = jobs_grid(a.jobs);
    const size_t js1 = smem_jobs_bytes(a.jobs);
    cudaError_t e = cudaSuccess;
    // with a body stream, the optional regions are IF nodes of the captured
    // graph (their kernels also check the control block themselves)
    auto open = [&](Gate which, int kernels) -> cudaStream_t {
        if (!body || e != cudaSuccess) return s;
        e = open_region(s, body, a.st, which, kernels);
        return body;
    };
    auto close = [&]() {
        if (body && e == cudaSuccess) e = close_region(body);
    };
    k_begin<<<jg, 256, 0, s>>>(a);
    if (prop0) {
        e = cudaEventRecordWithFlags(prop0, s, cudaEventRecordExternal);
        if (e != cudaSuccess) return e;
    }
    if (a.jobs == 1) {
        k_own<true><<<grid, kBlock, 0, s>>>(a);
        k_edges<true><<<grid, kBlock, 0, s>>>(a);
    } else {
        k_own<false><<<grid, kBlock, 0, s>>>(a);
        k_edges<false><<<grid, kBlock, 0, s>>>(a);
    }
    k_collect<<<grid, kBlock, js1, s>>>(a);
    if (prop1) {
        e = cudaEventRecordWithFlags(prop1, s, cudaEventRecordExternal);
        if (e != cudaSuccess) return e;
    }
    k_route<<<1, 1, 0, s>>>(a);
    {
        cudaStream_t r = open(kGateHeavy, 2 + kKernelsPerRebuild);
        if (e != cudaSuccess) return e;
        k_h_mark<<<g2, kBlock, js1, r>>>(a);
        k_h_apply<<<g2, kBlock, 0, r>>>(a, 0);
        e = launch_table_rebuild(a, rows, true, r, true);
        if (e != cudaSuccess) return e;
        close();
        if (e != cudaSuccess) return e;
    }
    {
        // second attempt of the heavy rebuild, when the tight capacity was
        // too small (the rebuild is still pending)
        cudaStream_t r = open(kGateRetry, kKernelsPerRebuild);
        if (e != cudaSuccess) return e;
        e = launch_table_rebuild(a, rows, true, r, true);
        if (e != cudaSuccess) return e;
        close();
        if (e != cudaSuccess) return e;
    }
    {
        cudaStream_t r = open(kGateHeavyEval, 2);
        if (e != cudaSuccess) return e;
        k_h_eval<<<g2, kBlock, js1, r>>>(a);
        k_h_decide<<<jg, 256, 0, r>>>(a);
        e = cudaGetLastError();
        close();
        if (e != cudaSuccess) return e;
    }
    {
        cudaStream_t r = open(kGateRollback, 1 + kKernelsPerRebuild);
        if (e != cudaSuccess) return e;
        k_h_apply<<<g2, kBlock, 0, r>>>(a, 1);
        e = launch_table_rebuild(a, rows, true, r);
        if (e != cudaSuccess) return e;
        close();
        if (e != cudaSuccess) return e;
    }
    {
        cudaStream_t r = open(kGateLight, 3);
        if (e != cudaSuccess) return e;
        k_stage<<<g2, kBlock, js1, r>>>(a);
        k_eval<<<g2, kBlock, js1, r>>>(a);
        k_decide<<<jg, 256, 0, r>>>(a);
        e = cudaGetLastError();
        close();
        if (e != cudaSuccess) return e;
    }
    k_bid<<<g2, kBlock, 0, s>>>(a);
    k_match_keys<<<g2, kBlock, 0, s>>>(a);
    k_commit<<<g2, kBlock, 2 * a.jobs <= kSmemJobs ? 2 * smem_jobs_bytes(a.jobs) : 0, s>>>(a);
    k_match_reset<<<g2, kBlock, 0, s>>>(a);
    k_end_jobs<<<jg, 256, 0, s>>>(a);
    k_end<<<1, 1, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    {
        cudaStream_t r = open(kGateRebuild, kKernelsPerRebuild);
        if (e != cudaSuccess) return e;
        e = launch_table_rebuild(a, rows, true, r);
        if (e != cudaSuccess) return e;
        close();
    }
    return e;
}

}  // namespace ccg
