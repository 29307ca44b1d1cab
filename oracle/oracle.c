/*
 * CPU oracle for median consensus clustering -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg use
 * this file.  It shares no code, header, table or helper with the CUDA path.
 * It is plain C: definitions written out, sorting and binary search as the
 * only "library" steps, no blocking or fusion.  Integer arithmetic throughout
 * (int64 for objectives and gains), so its results are exact.
 *
 * Notation (paper, Methods): n vertices, k input partitions P_1..P_k given as
 * labels[i*n + v] (partition-major), consensus C[v] = id of v's cluster.
 * Cluster ids are vertex ids in [0, n): the singleton start gives C[v] = v and
 * ids are never renumbered.
 *
 *   delta_uv          number of partitions separating u and v (Eq. rxyi, summed
 *                     over i; the printed P_k index is read as P_i)
 *   Mirkin(X, Y)      ordered pairs (u, v), u != v, co-clustered in exactly one
 *                     of X, Y (Methods: "counts (twice)"; Appendix Eq. distance
 *                     counts unordered pairs, i.e. half of this)
 *   F(C)              sum_i Mirkin(C, P_i)                         (Eq. objective1)
 *                   = k sum_c s_c^2 + sum_i sum_j |P_ij|^2 - 2 sum_{c,i,j} n(c,i,j)^2
 *   dD(v: a -> b)     sum_{u in a, u != v} (k - 2 delta_uv)
 *                     - sum_{u in b} (k - 2 delta_uv)        (Eq. objective3, u = v
 *                     excluded); the move changes F by exactly 2 dD.
 *                   = 2 (A_a - k - A_b) - k (|a| - 1 - |b|),
 *                     A_x = sum_i n(x, i, l_i(v))  (v counted in A_a)
 *
 * Synchronous sweep (Parallel algorithm section; the validation checks it
 * leaves open are fixed as follows):
 *   1. candidates of v: clusters of v's neighbours u != v, minus v's own
 *      cluster (Eq. objective4); an isolated vertex never moves;
 *   2. v proposes the candidate of least dD, ties to the smaller cluster id,
 *      and only if that dD < 0;  P = all proposals, against the sweep-start state;
 *   3. G1: a proposal between two singleton clusters a -> b survives only if
 *      b < a;  P1 = the survivors;
 *   4. G2: if P1 is non-empty and applying all of P1 at once lowers F, commit
 *      P1; otherwise commit the locally dominant matching of P: each cluster
 *      keeps the least key (dD, v) among the proposals that leave or enter it,
 *      and a proposal is committed iff it holds the least key at both its
 *      clusters;
 *   5. a sweep with no proposal ends the run, as does the sweep limit.
 * Move-to-empty variant (mode bit 2; not in the paper, whose candidate set
 * holds only clusters that contain a neighbour, Eq. objective4): v may also
 * move into a new cluster of its own, which takes the id v, provided no
 * vertex carries the id v at the sweep start (an id in use stays with its
 * cluster).  Its gain is Eq. objective3 with an empty target,
 *   dD(v: a -> {}) = sum_{u in a, u != v} (k - 2 delta_uv) = 2 (A_a - k) - k (|a| - 1),
 * and it competes with the neighbour candidates under the same (dD, id) rule;
 * the guards treat it like any other move (the singleton guard never applies:
 * the target is empty).
 * Colour-batched greedy (a variant between the two the Parallel algorithm
 * section contrasts -- all moves at once, one move at a time):
 *   colouring  priority(v) = splitmix64 of v (the first output of Steele, Lea
 *              and Flood's generator seeded with v: z = v + 0x9E3779B97F4A7C15,
 *              z = (z ^ z >> 30) * 0xBF58476D1CE4E5B9, z = (z ^ z >> 27) *
 *              0x94D049BB133111EB, z ^ z >> 31), a bijection, so priorities are
 *              distinct; in decreasing priority, each vertex takes the least
 *              colour that no neighbour coloured before it has (self-loops
 *              ignored).  Adjacent vertices get different colours.
 *   sweep      the colour classes c = 0, 1, ... in turn: the vertices of class c
 *              propose against the current state (candidates, ties, dD < 0 and
 *              the empty move if enabled as above) and the synchronous rule
 *              (steps 3-4) applies their proposals; the next class sees the
 *              result.  The sweep's record sums proposals, p1, dF_p1 and moves
 *              over the classes, counts the classes that fell back, and gives F
 *              after the last class.  A sweep with no proposal in any class ends
 *              the run, as does the sweep limit.
 * Sequential greedy (the one-move-at-a-time alternative the paper contrasts):
 * vertices in increasing index, each move evaluated on the current state and
 * applied at once if dD < 0, same candidate set and tie rule.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_INVALID 1
#define ORC_ERR_NOMEM 2

/* ---------------------------------------------------------------- helpers */

static int cmp_i32(const void* a, const void* b)
{
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* number of entries equal to key in a sorted int32 array (binary search) */
static int64_t count_sorted(const int32_t* arr, int64_t len, int32_t key)
{
    int64_t lo = 0, hi = len;
    while (lo < hi) { int64_t mid = lo + (hi - lo) / 2; if (arr[mid] < key) lo = mid + 1; else hi = mid; }
    int64_t first = lo;
    hi = len;
    while (lo < hi) { int64_t mid = lo + (hi - lo) / 2; if (arr[mid] <= key) lo = mid + 1; else hi = mid; }
    return lo - first;
}

/* sum of squared run lengths of a sorted array */
static int64_t sum_sq_runs(const int32_t* arr, int64_t len)
{
    int64_t s = 0, run = 0;
    for (int64_t p = 0; p < len; ++p) {
        if (p > 0 && arr[p] != arr[p - 1]) { s += run * run; run = 0; }
        ++run;
    }
    return s + run * run;
}

/* delta_uv: partitions in which u and v carry different labels (Eq. rxyi) */
static int64_t delta_uv(int32_t n, int32_t k, const int32_t* labels, int64_t u, int64_t v)
{
    int64_t d = 0;
    for (int32_t i = 0; i < k; ++i) d += labels[(int64_t)i * n + u] != labels[(int64_t)i * n + v];
    return d;
}

/* ------------------------------------------------------ contingency table
 * Members of every cluster listed contiguously (counting sort by cluster id,
 * vertices in increasing order), and for each partition i the members' labels
 * in that order, sorted inside each cluster's segment.  Then
 * n(x, i, l) = number of l in seg[i][start[x] .. start[x] + size[x]).        */
typedef struct {
    int32_t n, k;
    int64_t* start;   /* n + 1 */
    int32_t* size;    /* n */
    int32_t* members; /* n */
    int32_t* seg;     /* k * n */
} contingency;

static void ct_free(contingency* t)
{
    free(t->start); free(t->size); free(t->members); free(t->seg);
    memset(t, 0, sizeof(*t));
}

static int ct_build(contingency* t, int32_t n, int32_t k, const int32_t* labels, const int32_t* C)
{
    t->n = n; t->k = k;
    t->start = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    t->size = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
    t->members = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
    t->seg = (int32_t*)malloc(((size_t)k * n + 1) * sizeof(int32_t));
    if (!t->start || !t->size || !t->members || !t->seg) { ct_free(t); return ORC_ERR_NOMEM; }
    for (int32_t v = 0; v < n; ++v) {
        if (C[v] < 0 || C[v] >= n) { ct_free(t); return ORC_ERR_INVALID; }
        t->size[C[v]]++;
    }
    for (int32_t c = 0; c < n; ++c) t->start[c + 1] = t->start[c] + t->size[c];
    int64_t* fill = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!fill) { ct_free(t); return ORC_ERR_NOMEM; }
    memcpy(fill, t->start, (size_t)n * sizeof(int64_t));
    for (int32_t v = 0; v < n; ++v) t->members[fill[C[v]]++] = v;
    free(fill);
    #pragma omp parallel for schedule(dynamic, 1)
    for (int32_t i = 0; i < k; ++i) {
        int32_t* s = t->seg + (int64_t)i * n;
        const int32_t* l = labels + (int64_t)i * n;
        for (int32_t p = 0; p < n; ++p) s[p] = l[t->members[p]];
        for (int32_t c = 0; c < n; ++c)
            if (t->size[c] > 1) qsort(s + t->start[c], (size_t)t->size[c], sizeof(int32_t), cmp_i32);
    }
    return ORC_OK;
}

/* A_x(v) = sum_i n(x, i, l_i(v)) */
static int64_t ct_agree(const contingency* t, const int32_t* labels, int32_t x, int32_t v)
{
    int64_t a = 0;
    for (int32_t i = 0; i < t->k; ++i) {
        const int32_t* s = t->seg + (int64_t)i * t->n + t->start[x];
        a += count_sorted(s, t->size[x], labels[(int64_t)i * t->n + v]);
    }
    return a;
}

/* sum_{c,i,j} n(c,i,j)^2 */
static int64_t ct_sum_sq(const contingency* t)
{
    int64_t s = 0;
    for (int32_t i = 0; i < t->k; ++i)
        for (int32_t c = 0; c < t->n; ++c)
            if (t->size[c] > 0) s += sum_sq_runs(t->seg + (int64_t)i * t->n + t->start[c], t->size[c]);
    return s;
}

/* ---------------------------------------------------------- the objective */

/* sum_i sum_j |P_ij|^2 */
int64_t orc_partition_sq(int32_t n, int32_t k, const int32_t* labels)
{
    int32_t* tmp = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
    if (!tmp) return -1;
    int64_t s = 0;
    for (int32_t i = 0; i < k; ++i) {
        memcpy(tmp, labels + (int64_t)i * n, (size_t)n * sizeof(int32_t));
        qsort(tmp, (size_t)n, sizeof(int32_t), cmp_i32);
        s += n ? sum_sq_runs(tmp, n) : 0;
    }
    free(tmp);
    return s;
}

/* F(C) = k sum_c s_c^2 + sum_i sum_j |P_ij|^2 - 2 sum n(c,i,j)^2;  -1 on error */
int64_t orc_objective(int32_t n, int32_t k, const int32_t* labels, const int32_t* C)
{
    contingency t;
    if (ct_build(&t, n, k, labels, C) != ORC_OK) return -1;
    int64_t ss = 0;
    for (int32_t c = 0; c < n; ++c) ss += (int64_t)t.size[c] * t.size[c];
    int64_t F = (int64_t)k * ss + orc_partition_sq(n, k, labels) - 2 * ct_sum_sq(&t);
    ct_free(&t);
    return F;
}

/* Mirkin(X, Y) by enumerating ordered pairs (Appendix Eq. distance, doubled) */
int64_t orc_mirkin_pairs(int32_t n, const int32_t* X, const int32_t* Y)
{
    int64_t d = 0;
    for (int32_t u = 0; u < n; ++u)
        for (int32_t v = 0; v < n; ++v)
            if (u != v) d += (X[u] == X[v]) != (Y[u] == Y[v]);
    return d;
}

/* --------------------------------------------------------------- the gain */

/* dD(v: C[v] -> b) by iterating over members (Eq. objective3, u != v) */
int64_t orc_gain_member(int32_t n, int32_t k, const int32_t* labels, const int32_t* C, int32_t v, int32_t b)
{
    int32_t a = C[v];
    int64_t d = 0;
    for (int32_t u = 0; u < n; ++u) {
        if (u == v) continue;
        int64_t w = (int64_t)k - 2 * delta_uv(n, k, labels, u, v);
        if (C[u] == a) d += w;
        if (C[u] == b) d -= w;
    }
    return d;
}

/* dD(v: C[v] -> b) by the closed form, counts taken by a plain scan */
int64_t orc_gain_closed(int32_t n, int32_t k, const int32_t* labels, const int32_t* C, int32_t v, int32_t b)
{
    int32_t a = C[v];
    int64_t Aa = 0, Ab = 0, sa = 0, sb = 0;
    for (int32_t u = 0; u < n; ++u) {
        int64_t agree = (int64_t)k - delta_uv(n, k, labels, u, v);
        if (C[u] == a) { Aa += agree; ++sa; }
        if (C[u] == b) { Ab += agree; ++sb; }
    }
    return 2 * (Aa - k - Ab) - (int64_t)k * (sa - 1 - sb);
}

/* --------------------------------------------------- synchronous proposals */

/* mode bits: 1 = gains by member iteration (else from the contingency
 * table); 2 = the move-to-empty candidate */
#define ORC_MODE_MEMBER 1
#define ORC_MODE_EMPTY 2

/* gain of v -> x from the contingency table or by member iteration over the
 * cluster lists (x = -1: a new empty cluster) */
static int64_t sweep_gain(const contingency* t, int32_t n, int32_t k, const int32_t* labels,
                          int32_t v, int32_t a, int64_t Aa, int32_t x, int mode)
{
    if (!(mode & ORC_MODE_MEMBER)) {
        if (x < 0) return 2 * (Aa - k) - (int64_t)k * ((int64_t)t->size[a] - 1);
        int64_t Ax = ct_agree(t, labels, x, v);
        return 2 * (Aa - k - Ax) - (int64_t)k * ((int64_t)t->size[a] - 1 - t->size[x]);
    }
    int64_t d = 0;
    for (int64_t p = t->start[a]; p < t->start[a] + t->size[a]; ++p) {
        int32_t u = t->members[p];
        if (u != v) d += (int64_t)k - 2 * delta_uv(n, k, labels, u, v);
    }
    if (x < 0) return d;
    for (int64_t p = t->start[x]; p < t->start[x] + t->size[x]; ++p)
        d -= (int64_t)k - 2 * delta_uv(n, k, labels, t->members[p], v);
    return d;
}

/* Best move of every vertex against state C (Eq. objective4).  target[v] = -1
 * when v does not propose.  Returns the number of proposals, -1 on error. */
static int64_t sync_propose_range(const contingency* t, int32_t n, const int64_t* row_off, const int32_t* col,
                                  int32_t k, const int32_t* labels, const int32_t* C,
                                  int32_t* target, int64_t* gain, int mode, int32_t v0, int32_t v1,
                                  const int32_t* cls, int32_t c);

static int64_t sync_propose(const contingency* t, int32_t n, const int64_t* row_off, const int32_t* col,
                            int32_t k, const int32_t* labels, const int32_t* C,
                            int32_t* target, int64_t* gain, int mode)
{
    return sync_propose_range(t, n, row_off, col, k, labels, C, target, gain, mode, 0, n, NULL, 0);
}

/* The proposals of the vertices v0 <= v < v1 only, and (cls not NULL) only
 * of those with cls[v] == c; the others get no proposal. */
static int64_t sync_propose_range(const contingency* t, int32_t n, const int64_t* row_off, const int32_t* col,
                                  int32_t k, const int32_t* labels, const int32_t* C,
                                  int32_t* target, int64_t* gain, int mode, int32_t v0, int32_t v1,
                                  const int32_t* cls, int32_t c)
{
    int32_t maxdeg = 0;
    for (int32_t v = 0; v < n; ++v) {
        int64_t d = row_off[v + 1] - row_off[v];
        if (d > maxdeg) maxdeg = (int32_t)d;
    }
    int64_t count = 0;
    int failed = 0;
    #pragma omp parallel reduction(+:count)
    {
        int32_t* cand = (int32_t*)malloc(((size_t)maxdeg + 1) * sizeof(int32_t));
        if (!cand) {
            #pragma omp atomic write
            failed = 1;
        }
        #pragma omp for schedule(dynamic, 64)
        for (int32_t v = 0; v < n; ++v) {
            target[v] = -1;
            gain[v] = 0;
            if (!cand || v < v0 || v >= v1 || (cls && cls[v] != c)) continue;
            int32_t a = C[v];
            int64_t m = 0;
            for (int64_t e = row_off[v]; e < row_off[v + 1]; ++e) {
                int32_t u = col[e];
                if (u == v || C[u] == a) continue;
                cand[m++] = C[u];
            }
            /* the empty cluster with id v, if that id is free */
            const int empty = (mode & ORC_MODE_EMPTY) && t->size[v] == 0;
            if (m == 0 && !empty) continue;
            qsort(cand, (size_t)m, sizeof(int32_t), cmp_i32);
            int64_t Aa = (mode & ORC_MODE_MEMBER) ? 0 : ct_agree(t, labels, a, v);
            int64_t best = 0;
            int32_t best_x = -1;
            for (int64_t j = 0; j < m; ++j) {
                if (j > 0 && cand[j] == cand[j - 1]) continue;
                int64_t g = sweep_gain(t, n, k, labels, v, a, Aa, cand[j], mode);
                if (best_x < 0 || g < best) { best = g; best_x = cand[j]; }  /* ascending ids: ties keep the smaller */
            }
            if (empty) {
                int64_t g = sweep_gain(t, n, k, labels, v, a, Aa, -1, mode);
                if (best_x < 0 || g < best || (g == best && v < best_x)) { best = g; best_x = v; }
            }
            if (best < 0) { target[v] = best_x; gain[v] = best; ++count; }
        }
        free(cand);
    }
    return failed ? -1 : count;
}

/* Locally dominant matching of a proposal set (target[v] >= 0 means v
 * proposes C[v] -> target[v] with gain[v]): every cluster keeps the least key
 * (gain, v), compared lexicographically, among the proposals that leave or
 * enter it; v is kept (moved[v] = 1) iff it holds the least key at both of its
 * clusters.  Returns the number kept, -1 on allocation failure. */
int64_t orc_match(int32_t n, const int32_t* C, const int32_t* target, const int64_t* gain, int32_t* moved)
{
    int64_t* bg = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
    int32_t* bv = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
    if (!bg || !bv) { free(bg); free(bv); return -1; }
    for (int32_t x = 0; x < n; ++x) { bg[x] = 0; bv[x] = -1; }
    for (int32_t v = 0; v < n; ++v) {
        if (target[v] < 0) continue;
        int32_t ends[2] = { C[v], target[v] };
        for (int e = 0; e < 2; ++e) {
            int32_t x = ends[e];
            if (bv[x] < 0 || gain[v] < bg[x] || (gain[v] == bg[x] && v < bv[x])) { bg[x] = gain[v]; bv[x] = v; }
        }
    }
    int64_t kept = 0;
    for (int32_t v = 0; v < n; ++v) {
        moved[v] = target[v] >= 0 && bv[C[v]] == v && bv[target[v]] == v;
        kept += moved[v];
    }
    free(bg); free(bv);
    return kept;
}

typedef struct {
    int64_t proposals;   /* |P| */
    int64_t p1;          /* |P1| after the singleton guard */
    int64_t dF_p1;       /* F(C with P1 applied) - F(C); 0 when P1 is empty */
    int64_t fallback;    /* 1 when the matching was committed */
    int64_t moves;       /* moves committed */
    int64_t F;           /* F after the sweep */
} orc_sweep_stats;

/* Proposals of one sweep against state C (for tests). */
int64_t orc_sync_propose(int32_t n, const int64_t* row_off, const int32_t* col, int32_t k,
                         const int32_t* labels, const int32_t* C, int32_t* target, int64_t* gain,
                         int32_t mode, int32_t threads)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
    (void)threads;
    contingency t;
    if (ct_build(&t, n, k, labels, C) != ORC_OK) return -1;
    int64_t r = sync_propose(&t, n, row_off, col, k, labels, C, target, gain, mode);
    ct_free(&t);
    return r;
}

/* Proposals of the vertices in [v0, v1) against state C (the others: none). */
int64_t orc_sync_propose_range(int32_t n, const int64_t* row_off, const int32_t* col, int32_t k,
                               const int32_t* labels, const int32_t* C, int32_t v0, int32_t v1,
                               int32_t* target, int64_t* gain, int32_t mode, int32_t threads)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
    (void)threads;
    contingency t;
    if (ct_build(&t, n, k, labels, C) != ORC_OK) return -1;
    int64_t r = sync_propose_range(&t, n, row_off, col, k, labels, C, target, gain, mode, v0, v1, NULL, 0);
    ct_free(&t);
    return r;
}

static int32_t sync_step_class(int32_t n, const int64_t* row_off, const int32_t* col, int32_t k,
                               const int32_t* labels, int32_t* C, int64_t F_in, int32_t mode,
                               orc_sweep_stats* st, int32_t* target_out, int64_t* gain_out, int32_t* moved_out,
                               const int32_t* cls, int32_t c);

/* One synchronous sweep on C (in/out).  F_in = F(C).  Optional per-vertex
 * outputs: the proposals of this sweep (target, gain) and which vertices moved. */
int32_t orc_sync_step(int32_t n, const int64_t* row_off, const int32_t* col, int32_t k,
                      const int32_t* labels, int32_t* C, int64_t F_in, int32_t mode,
                      orc_sweep_stats* st, int32_t* target_out, int64_t* gain_out, int32_t* moved_out)
{
    return sync_step_class(n, row_off, col, k, labels, C, F_in, mode, st, target_out, gain_out, moved_out, NULL, 0);
}

/* The synchronous rule applied to the proposals of the vertices with
 * cls[v] == c (all vertices when cls is NULL). */
static int32_t sync_step_class(int32_t n, const int64_t* row_off, const int32_t* col, int32_t k,
                               const int32_t* labels, int32_t* C, int64_t F_in, int32_t mode,
                               orc_sweep_stats* st, int32_t* target_out, int64_t* gain_out, int32_t* moved_out,
                               const int32_t* cls, int32_t c)
{
    memset(st, 0, sizeof(*st));
    contingency t;
    if (ct_build(&t, n, k, labels, C) != ORC_OK) return ORC_ERR_INVALID;
    int32_t* target = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
    int64_t* gain = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
    int32_t* C1 = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
    int32_t* moved = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
    if (!target || !gain || !C1 || !moved) {
        free(target); free(gain); free(C1); free(moved); ct_free(&t); return ORC_ERR_NOMEM;
    }
    int64_t np = sync_propose_range(&t, n, row_off, col, k, labels, C, target, gain, mode, 0, n, cls, c);
    st->proposals = np < 0 ? 0 : np;
    st->F = F_in;
    if (np > 0) {
        /* G1: singleton -> singleton only towards the smaller id */
        memcpy(C1, C, (size_t)n * sizeof(int32_t));
        int64_t p1 = 0;
        for (int32_t v = 0; v < n; ++v) {
            if (target[v] < 0) continue;
            int32_t a = C[v], b = target[v];
            int both_single = t.size[a] == 1 && t.size[b] == 1;
            if (!both_single || b < a) { C1[v] = b; ++p1; }
        }
        st->p1 = p1;
        int64_t F1 = F_in;
        if (p1 > 0) {
            F1 = orc_objective(n, k, labels, C1);   /* G2: the exact F after applying P1 at once */
            st->dF_p1 = F1 - F_in;
        }
        if (p1 > 0 && st->dF_p1 < 0) {
            for (int32_t v = 0; v < n; ++v) if (C1[v] != C[v]) moved[v] = 1;
            memcpy(C, C1, (size_t)n * sizeof(int32_t));
            st->moves = p1;
            st->F = F1;
        } else {
            /* locally dominant matching over all of P */
            int64_t moves = orc_match(n, C, target, gain, moved);
            if (moves < 0) { free(target); free(gain); free(C1); free(moved); ct_free(&t); return ORC_ERR_NOMEM; }
            for (int32_t v = 0; v < n; ++v) if (moved[v]) C[v] = target[v];
            st->fallback = 1;
            st->moves = moves;
            st->F = orc_objective(n, k, labels, C);
        }
    }
    if (target_out) memcpy(target_out, target, (size_t)n * sizeof(int32_t));
    if (gain_out) memcpy(gain_out, gain, (size_t)n * sizeof(int64_t));
    if (moved_out) memcpy(moved_out, moved, (size_t)n * sizeof(int32_t));
    free(target); free(gain); free(C1); free(moved);
    ct_free(&t);
    return ORC_OK;
}

/* Runs synchronous sweeps from C (in/out; pass C[v] = v for the singleton
 * start) until a sweep has no proposal or max_sweeps sweeps ran.
 * stats must hold max_sweeps entries; *sweeps_done counts every sweep run,
 * the final empty one included. */
int32_t orc_sync_run(int32_t n, const int64_t* row_off, const int32_t* col, int32_t k,
                     const int32_t* labels, int32_t* C, int32_t max_sweeps, int32_t mode,
                     int32_t threads, orc_sweep_stats* stats, int32_t* sweeps_done)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
    (void)threads;
    *sweeps_done = 0;
    int64_t F = orc_objective(n, k, labels, C);
    if (F < 0) return ORC_ERR_INVALID;
    for (int32_t s = 0; s < max_sweeps; ++s) {
        int32_t rc = orc_sync_step(n, row_off, col, k, labels, C, F, mode, &stats[s], NULL, NULL, NULL);
        if (rc != ORC_OK) return rc;
        *sweeps_done = s + 1;
        F = stats[s].F;
        if (stats[s].proposals == 0) break;
    }
    return ORC_OK;
}

/* ------------------------------------------------- colour-batched greedy */

/* Priority of vertex v: the first output of splitmix64 seeded with v. */
uint64_t orc_priority(uint64_t v)
{
    uint64_t z = v + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

typedef struct { uint64_t p; int32_t v; } orc_prio;

static int cmp_prio_desc(const void* a, const void* b)
{
    uint64_t x = ((const orc_prio*)a)->p, y = ((const orc_prio*)b)->p;
    return (x < y) - (x > y);
}

/* Greedy colouring in decreasing priority; colour[v] written; returns the
 * number of colours, -1 on allocation failure. */
int32_t orc_colour(int32_t n, const int64_t* row_off, const int32_t* col, int32_t* colour)
{
    orc_prio* order = (orc_prio*)malloc(((size_t)n + 1) * sizeof(orc_prio));
    int32_t maxdeg = 0;
    for (int32_t v = 0; v < n; ++v) {
        int64_t d = row_off[v + 1] - row_off[v];
        if (d > maxdeg) maxdeg = (int32_t)d;
    }
    uint8_t* used = (uint8_t*)calloc((size_t)maxdeg + 2, 1);
    if (!order || !used) { free(order); free(used); return -1; }
    for (int32_t v = 0; v < n; ++v) { order[v].p = orc_priority((uint64_t)v); order[v].v = v; colour[v] = -1; }
    qsort(order, (size_t)n, sizeof(orc_prio), cmp_prio_desc);
    int32_t colours = 0;
    for (int32_t r = 0; r < n; ++r) {
        int32_t v = order[r].v;
        for (int64_t e = row_off[v]; e < row_off[v + 1]; ++e) {
            int32_t u = col[e], cu = u != v ? colour[u] : -1;
            if (cu >= 0 && cu <= maxdeg) used[cu] = 1;
        }
        int32_t c = 0;
        while (used[c]) ++c;
        colour[v] = c;
        if (c + 1 > colours) colours = c + 1;
        for (int64_t e = row_off[v]; e < row_off[v + 1]; ++e) {
            int32_t u = col[e], cu = u != v ? colour[u] : -1;
            if (cu >= 0 && cu <= maxdeg) used[cu] = 0;
        }
    }
    free(order); free(used);
    return colours;
}

/* Colour-batched greedy sweeps from C (in/out) with the colouring colour[]
 * (as orc_colour gives it; `colours` classes), until a sweep has no proposal
 * or max_sweeps sweeps ran.  stats as orc_sync_run. */
int32_t orc_colour_run(int32_t n, const int64_t* row_off, const int32_t* col, int32_t k,
                       const int32_t* labels, int32_t* C, const int32_t* colour, int32_t colours,
                       int32_t max_sweeps, int32_t mode, int32_t threads, orc_sweep_stats* stats,
                       int32_t* sweeps_done)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
    (void)threads;
    *sweeps_done = 0;
    int64_t F = orc_objective(n, k, labels, C);
    if (F < 0) return ORC_ERR_INVALID;
    for (int32_t s = 0; s < max_sweeps; ++s) {
        orc_sweep_stats tot;
        memset(&tot, 0, sizeof(tot));
        for (int32_t c = 0; c < colours; ++c) {
            orc_sweep_stats st;
            int32_t rc = sync_step_class(n, row_off, col, k, labels, C, F, mode, &st, NULL, NULL, NULL, colour, c);
            if (rc != ORC_OK) return rc;
            tot.proposals += st.proposals;
            tot.p1 += st.p1;
            tot.dF_p1 += st.dF_p1;
            tot.fallback += st.fallback;
            tot.moves += st.moves;
            F = st.F;
        }
        tot.F = F;
        stats[s] = tot;
        *sweeps_done = s + 1;
        if (tot.proposals == 0) break;
    }
    return ORC_OK;
}

/* ----------------------------------------------------- sequential greedy
 * Counts n(x, i, l) kept in a plain open-addressing map keyed by (x, i, l). */
typedef struct { int32_t x, i, l, used; int64_t cnt; } seq_slot;

static uint64_t seq_hash(int32_t x, int32_t i, int32_t l)
{
    uint64_t h = (uint64_t)(uint32_t)x * 0x9E3779B97F4A7C15ull;
    h ^= (uint64_t)(uint32_t)i * 0xC2B2AE3D27D4EB4Full + (h << 6) + (h >> 2);
    h ^= (uint64_t)(uint32_t)l * 0x165667B19E3779F9ull + (h << 6) + (h >> 2);
    return h ^ (h >> 29);
}

static seq_slot* seq_find(seq_slot* tab, uint64_t mask, int32_t x, int32_t i, int32_t l, int insert)
{
    uint64_t h = seq_hash(x, i, l) & mask;
    for (uint64_t p = 0; p <= mask; ++p, h = (h + 1) & mask) {
        seq_slot* s = &tab[h];
        if (!s->used) {
            if (!insert) return NULL;
            s->used = 1; s->x = x; s->i = i; s->l = l; s->cnt = 0;
            return s;
        }
        if (s->x == x && s->i == i && s->l == l) return s;
    }
    return NULL;
}

/* Sequential greedy from C (in/out).  F_trace[s] = F after sweep s,
 * moves_trace[s] = moves in sweep s.  Returns ORC_OK or an error. */
int32_t orc_seq_run(int32_t n, const int64_t* row_off, const int32_t* col, int32_t k,
                    const int32_t* labels, int32_t* C, int32_t max_sweeps,
                    int64_t* F_trace, int64_t* moves_trace, int32_t* sweeps_done)
{
    *sweeps_done = 0;
    int64_t F = orc_objective(n, k, labels, C);
    if (F < 0) return ORC_ERR_INVALID;
    uint64_t cap = 1;
    while (cap < 4 * (uint64_t)k * (uint64_t)n + 16) cap <<= 1;
    seq_slot* tab = (seq_slot*)calloc(cap, sizeof(seq_slot));
    int32_t* size = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
    int32_t maxdeg = 0;
    for (int32_t v = 0; v < n; ++v) if (row_off[v + 1] - row_off[v] > maxdeg) maxdeg = (int32_t)(row_off[v + 1] - row_off[v]);
    int32_t* cand = (int32_t*)malloc(((size_t)maxdeg + 1) * sizeof(int32_t));
    if (!tab || !size || !cand) { free(tab); free(size); free(cand); return ORC_ERR_NOMEM; }
    for (int32_t v = 0; v < n; ++v) {
        size[C[v]]++;
        for (int32_t i = 0; i < k; ++i) seq_find(tab, cap - 1, C[v], i, labels[(int64_t)i * n + v], 1)->cnt++;
    }
    for (int32_t s = 0; s < max_sweeps; ++s) {
        int64_t moves = 0;
        for (int32_t v = 0; v < n; ++v) {
            int32_t a = C[v];
            int64_t m = 0;
            for (int64_t e = row_off[v]; e < row_off[v + 1]; ++e) {
                int32_t u = col[e];
                if (u != v && C[u] != a) cand[m++] = C[u];
            }
            if (m == 0) continue;
            qsort(cand, (size_t)m, sizeof(int32_t), cmp_i32);
            int64_t Aa = 0;
            for (int32_t i = 0; i < k; ++i) Aa += seq_find(tab, cap - 1, a, i, labels[(int64_t)i * n + v], 0)->cnt;
            int64_t best = 0;
            int32_t bx = -1;
            for (int64_t j = 0; j < m; ++j) {
                if (j > 0 && cand[j] == cand[j - 1]) continue;
                int32_t x = cand[j];
                int64_t Ax = 0;
                for (int32_t i = 0; i < k; ++i) {
                    seq_slot* sl = seq_find(tab, cap - 1, x, i, labels[(int64_t)i * n + v], 0);
                    if (sl) Ax += sl->cnt;
                }
                int64_t g = 2 * (Aa - k - Ax) - (int64_t)k * ((int64_t)size[a] - 1 - size[x]);
                if (bx < 0 || g < best) { best = g; bx = x; }
            }
            if (best < 0) {
                for (int32_t i = 0; i < k; ++i) {
                    int32_t l = labels[(int64_t)i * n + v];
                    seq_find(tab, cap - 1, a, i, l, 0)->cnt--;
                    seq_slot* sl = seq_find(tab, cap - 1, bx, i, l, 1);
                    if (!sl) { free(tab); free(size); free(cand); return ORC_ERR_NOMEM; }
                    sl->cnt++;
                }
                size[a]--; size[bx]++;
                C[v] = bx;
                F += 2 * best;
                ++moves;
            }
        }
        F_trace[s] = F;
        moves_trace[s] = moves;
        *sweeps_done = s + 1;
        if (moves == 0) break;
    }
    free(tab); free(size); free(cand);
    return ORC_OK;
}

/* ------------------------------------------------------------ brute force
 * Exact optimum of F over all set partitions of n <= 12 vertices, by
 * enumerating restricted growth strings; F counted pair by pair. */
int64_t orc_brute_force(int32_t n, int32_t k, const int32_t* labels, int32_t* best_C)
{
    if (n < 1 || n > 12) return -1;
    int64_t delta[12][12];
    for (int32_t u = 0; u < n; ++u)
        for (int32_t v = 0; v < n; ++v) delta[u][v] = delta_uv(n, k, labels, u, v);
    int32_t rgs[12] = {0}, mx[12] = {0};
    int64_t best = -1;
    for (;;) {
        int64_t F = 0;
        for (int32_t u = 0; u < n; ++u)
            for (int32_t v = 0; v < n; ++v)
                if (u != v) F += rgs[u] == rgs[v] ? delta[u][v] : (int64_t)k - delta[u][v];
        if (best < 0 || F < best) {
            best = F;
            if (best_C) for (int32_t v = 0; v < n; ++v) best_C[v] = rgs[v];
        }
        int32_t j = n - 1;   /* next restricted growth string */
        while (j > 0 && rgs[j] > mx[j - 1]) --j;
        if (j == 0) break;
        rgs[j]++;
        mx[j] = rgs[j] > mx[j - 1] ? rgs[j] : mx[j - 1];
        for (int32_t q = j + 1; q < n; ++q) { rgs[q] = 0; mx[q] = mx[j]; }
    }
    return best;
}

/* ------------------------------------------------ partition comparison */
/*
 * Distances between a partition C and each input partition P_i (Methods,
 * "Evaluation metrics": the paper compares partitions by the Rand distance,
 * the split-join distance and the variation of information; it states no
 * formulas, so the standard definitions are written out here):
 *   mirkin[i]      Mirkin(C, P_i) over ordered pairs (the Rand distance is
 *                  mirkin / (n (n - 1)));
 *   split_join[i]  van Dongen's split-join distance: 2n - sum over clusters c
 *                  of C of max_l |c & l| - sum over classes l of P_i of
 *                  max_c |c & l|;
 *   vi[i]          Meila's variation of information H(C | P_i) + H(P_i | C)
 *                  in nats, with p(c, l) = |c & l| / n:
 *                  - sum_{c,l} p(c,l) [log(p(c,l) / p(l)) + log(p(c,l) / p(c))].
 * The contingency of (C, P_i) comes from sorting the pairs (c, l) of all
 * vertices; sizes of c and l from sorting C and the labels.
 */
static int cmp_u64(const void* a, const void* b)
{
    const uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return x < y ? -1 : x > y;
}

/* Count of x in the sorted array (binary search for the run). */
static int64_t run_of(const int32_t* arr, int64_t len, int32_t x)
{
    return count_sorted(arr, len, x);
}

int32_t orc_metrics(int32_t n, int32_t k, const int32_t* labels, const int32_t* C, int64_t* mirkin,
                    int64_t* split_join, double* vi)
{
    uint64_t* cl = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));  /* (c, l) pairs */
    uint64_t* lc = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));  /* (l, c) pairs */
    int32_t* cs = (int32_t*)malloc((size_t)n * sizeof(int32_t));     /* sorted C */
    int32_t* ls = (int32_t*)malloc((size_t)n * sizeof(int32_t));     /* sorted labels */
    if (!cl || !lc || !cs || !ls) { free(cl); free(lc); free(cs); free(ls); return ORC_ERR_NOMEM; }
    memcpy(cs, C, (size_t)n * sizeof(int32_t));
    qsort(cs, (size_t)n, sizeof(int32_t), cmp_i32);
    for (int32_t i = 0; i < k; ++i) {
        const int32_t* L = labels + (int64_t)i * n;
        for (int32_t v = 0; v < n; ++v) {
            /* order-preserving 32-bit images of the two ids */
            const uint64_t c = (uint32_t)C[v] ^ 0x80000000u, l = (uint32_t)L[v] ^ 0x80000000u;
            cl[v] = (c << 32) | l;
            lc[v] = (l << 32) | c;
            ls[v] = L[v];
        }
        qsort(cl, (size_t)n, sizeof(uint64_t), cmp_u64);
        qsort(lc, (size_t)n, sizeof(uint64_t), cmp_u64);
        qsort(ls, (size_t)n, sizeof(int32_t), cmp_i32);
        int64_t sq = 0, max_over_l = 0, max_over_c = 0;
        double h = 0.0;
        /* runs of equal (c, l): n(c, l); the best run within each c */
        for (int64_t a = 0, best = 0; a < n;) {
            int64_t b = a;
            while (b < n && cl[b] == cl[a]) ++b;
            const int64_t ncl = b - a;
            sq += ncl * ncl;
            const int32_t c = (int32_t)((uint32_t)(cl[a] >> 32) ^ 0x80000000u);
            const int32_t l = (int32_t)((uint32_t)cl[a] ^ 0x80000000u);
            const double p = (double)ncl / n;
            const double pc = (double)run_of(cs, n, c) / n, pl = (double)run_of(ls, n, l) / n;
            h -= p * (log(p / pl) + log(p / pc));
            if (ncl > best) best = ncl;
            if (b == n || (cl[b] >> 32) != (cl[a] >> 32)) {
                max_over_l += best;
                best = 0;
            }
            a = b;
        }
        /* the best run within each l */
        for (int64_t a = 0, best = 0; a < n;) {
            int64_t b = a;
            while (b < n && lc[b] == lc[a]) ++b;
            if (b - a > best) best = b - a;
            if (b == n || (lc[b] >> 32) != (lc[a] >> 32)) {
                max_over_c += best;
                best = 0;
            }
            a = b;
        }
        mirkin[i] = sum_sq_runs(cs, n) + sum_sq_runs(ls, n) - 2 * sq;
        split_join[i] = 2 * (int64_t)n - max_over_l - max_over_c;
        vi[i] = h;
    }
    free(cl); free(lc); free(cs); free(ls);
    return ORC_OK;
}
