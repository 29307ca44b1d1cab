/*
 * cc.h -- C ABI of the GB300 median-consensus sweep library (libcc.so).
 *
 * Method: graph-aware median consensus clustering (Hussain, Halappanavar,
 * Chatterjee, Radicchi, Fortunato, Azad, "Parallel Algorithms for Median
 * Consensus Clustering in Complex Networks", arXiv 2408.11331).  Given a graph
 * and k input partitions P_1..P_k of its n vertices, the library starts from
 * singleton clusters and runs synchronous greedy local-move sweeps that lower
 * F(C) = sum_i Mirkin(C, P_i) (Eq. objective1), each vertex considering only
 * the clusters of its neighbours (Eq. objective4) and scored by the exact
 * integer change of Eq. objective3.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Host pointers are borrowed for the duration of the call and copied; the
 *   library never keeps them.  The _dev variants take device pointers under the
 *   same rule.  All output buffers are caller-allocated.
 * - The context owns every device buffer it allocates and frees them in
 *   cc_destroy.  All device work of a context runs on one CUDA stream (its
 *   own, or the one given to cc_set_stream); entry points that return host
 *   values synchronise that stream.
 * - Every call returns a cc_status; nothing is thrown across the ABI.  After a
 *   failure, cc_last_error(ctx) describes it.  CC_ERR_CUDA leaves the context
 *   unusable; the other errors leave it as it was before the call.
 * - Objective values use ordered pairs (the Mirkin distance counts each
 *   disagreeing pair twice, Methods); the unordered count is F / 2.
 * - Cluster ids are founding-vertex ids: the singleton start gives C[v] = v and
 *   ids are never renumbered, because ties between candidates go to the
 *   smaller id.
 * - Arithmetic is integer and exact.  Gains are int32, which requires
 *   3 k n + k < 2^31 (else CC_ERR_OVERFLOW); objectives are int64.
 * - Not thread-safe per context; distinct contexts may be used concurrently.
 */
#ifndef CC_H
#define CC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cc_ctx cc_ctx;

typedef enum {
    CC_OK = 0,
    CC_ERR_INVALID = 1,    /* malformed argument: null pointer, n < 1, k < 1, nnz < 0, CSR offsets
                              not starting at 0 / not ending at nnz / decreasing, column out of range */
    CC_ERR_OOM = 2,        /* a device allocation failed */
    CC_ERR_CUDA = 3,       /* a CUDA runtime call or kernel failed */
    CC_ERR_OVERFLOW = 4,   /* 3 k n + k >= 2^31: an int32 gain could overflow */
    CC_ERR_TABLE_FULL = 5, /* the contingency hash ran out of slots (bounded probing gave up) */
    CC_ERR_TIMEOUT = 6     /* reserved: a bounded device wait gave up */
} cc_status;

typedef struct {
    int32_t max_sweeps;     /* sweep limit used when cc_run_until_converged gets max_sweeps <= 0;
                               default 20 */
    int32_t debug_checks;   /* 1: after every sweep recompute F from scratch on the device and
                               fail with CC_ERR_INVALID if it differs from the incremental F */
    int32_t table_log2;     /* log2 of the allocated contingency hash capacity (slots of 16
                               bytes); 0 = automatic: the least power of two >= 2 k n + 64
                               (>= 4 k n + 64 with sweep_mode 1) */
    int32_t table_start_log2; /* log2 of the capacity in use at the singleton start; 0 =
                               automatic (>= 2 k n).  The capacity in use then follows the
                               live keys; a sweep that would fill it is abandoned before
                               it commits anything and retried in twice the capacity */
    int32_t sweep_mode;     /* how a sweep evaluates dF of its kept moves P1 (the results are
                               identical): 0 = automatic (a rebuild of the contingency hash
                               from the tentatively moved consensus when more than n/8
                               vertices propose -- in a batch, when the proposals carry more
                               than 1/8 of all label rows -- otherwise staged count
                               deltas); 1 = always
                               staged deltas (the hash is built at the singleton start);
                               2 = always a rebuild */
    int32_t lanes;          /* lanes of a warp that score one candidate move, one proposal of the
                               light path or one vertex's own cluster: 1, 2, 4, 8, 16 or 32;
                               0 = automatic (by the largest k: about 10 partitions per lane).
                               Results do not depend on it; speed does */
    int32_t active_set;     /* 1: after the first sweep of a run, a vertex whose own cluster and
                               whose previous bid's target did not change in the previous
                               sweep scores only its candidates whose cluster changed and
                               keeps its previous bid if that stays the least (exactly what
                               scoring every candidate would give).  Results are identical;
                               it changes how many edges a sweep evaluates.  0 (default):
                               every sweep scores every edge */
    int32_t no_regions;     /* 1: capture every kernel of a sweep as a plain node of the sweep
                               graph (a region a sweep does not need runs kernels that return at
                               once) instead of behind conditional nodes; for profilers that
                               cannot see kernels inside graphs with conditional nodes.  Results
                               are identical.  0 (default): conditional regions */
    int32_t empty_moves;    /* 1: the move-to-empty variant.  Besides the clusters of its
                               neighbours (Eq. objective4), a vertex v may move into a new
                               cluster of its own, which takes the id v, provided no vertex
                               carries the id v at the start of the sweep.  Its gain is Eq.
                               objective3 with an empty target, sum over u in a, u != v, of
                               (k - 2 delta_uv) = 2 (A_a - k) - k (|a| - 1), and it competes
                               with the other candidates under the same rule (least dD, ties to
                               the smaller id).  This changes the results (a quality variant the
                               paper does not consider).  0 (default): the paper's candidates */
    int32_t colour_batched; /* 1: the colour-batched variant, between the paper's two (all moves
                               at once, one move at a time; Parallel algorithm section).  The
                               graph is coloured once: in decreasing priority (the first
                               splitmix64 output seeded with the job-local vertex id) each vertex
                               takes the least colour no earlier-coloured neighbour has, so
                               adjacent vertices differ.  A sweep then runs the colour classes in
                               turn: the vertices of one class propose against the current state
                               and the synchronous rule (guards, matching) applies them, so each
                               class sees the moves of the classes before it.  A sweep's record
                               sums the classes (fallback: classes that fell back); the run stops
                               after a sweep without any proposal.  Changes the results.  Needs
                               active_set = 0 and fewer than 2^31 CSR entries per context.
                               cc_last_run_timing then gives one entry per class run.  0
                               (default): the synchronous sweep */
    int32_t autotune;       /* 1 (with lanes = 0): the first run of the context times its
                               proposal kernels once for each candidate lane count (the
                               automatic choice, half and twice it) on the state after the run's
                               first sweep, and keeps the fastest; the choice is remembered per
                               device and lane bin (see cc_plan_batches) for the later contexts
                               of the process, which then skip the timing.  Results are
                               identical; only speed changes.  0 (default): automatic rule */
    int32_t tight_rebuild;  /* Capacity of the rebuild of a heavy sweep (results are identical
                               for every value).  0 (default): first a tight capacity, from
                               the occupied slots at the sweep start at load <= 1/2 with room
                               for a following light sweep; a build that does not fit it (an
                               insert past 256 probes, load above 1/2, or too little room) is
                               dropped and redone at the capacity that holds every key the
                               sweep can create.  1: always that safe capacity.  2: the tight
                               attempt is always dropped (for tests of the second attempt) */
} cc_options;

/* State of the contingency hash of a context. */
typedef struct {
    int64_t capacity;      /* slots in use (a power of two) */
    int64_t max_capacity;  /* slots allocated */
    int64_t live_keys;     /* (cluster, partition, label) keys with a non-zero count */
    int64_t used_slots;    /* occupied slots, dead keys included */
    int64_t rebuilds;      /* rebuilds since creation (reset included) */
    int64_t retries;       /* sweeps abandoned for lack of space and run again */
} cc_table_info;

/* Per-sweep record.  Field meanings follow the synchronous sweep of the
 * Parallel algorithm section with its validation checks fixed as:
 *   proposals  |P|: vertices whose best graph-restricted move (Eq. objective4)
 *              has dD < 0 against the sweep-start state (ties: smaller id)
 *   p1         |P1|: proposals kept by the singleton guard (a move between two
 *              singleton clusters a -> b is kept only if b < a)
 *   dF_p1      exact F(C with all of P1 applied) - F(C); 0 when P1 is empty
 *   fallback   1 if P1 was empty or dF_p1 >= 0 and the locally dominant
 *              matching of P was committed instead (each cluster keeps the
 *              least (dD, v) of the proposals leaving or entering it; a move is
 *              committed iff it holds the least key at both its clusters)
 *   moves      moves committed
 *   F          objective after the sweep                                     */
typedef struct {
    int64_t proposals;
    int64_t p1;
    int64_t dF_p1;
    int64_t fallback;
    int64_t moves;
    int64_t F;
} cc_sweep_info;

/* Fills *opt with the defaults (max_sweeps 20, no debug checks, automatic
 * table size).  Never fails for a non-null opt. */
void cc_default_options(cc_options* opt);

/* Creates a context for one consensus job and puts it at the singleton start
 * (The algorithm: Initialization).
 *   n        number of vertices, >= 1
 *   nnz      number of CSR entries, >= 0 (an undirected edge appears twice)
 *   row_off  int64[n + 1] host, row_off[0] = 0, non-decreasing, row_off[n] = nnz
 *   col      int32[nnz]   host, neighbour ids in [0, n); self-loops and repeated
 *            entries are allowed and ignored (candidate sets are sets)
 *   k        number of input partitions, >= 1
 *   labels   int32[k * n] host, partition-major: labels[i * n + v] is v's
 *            cluster in P_i; any int32 values, only equality matters
 *   opt      options, or NULL for the defaults
 *   out      receives the new context; set to NULL on failure
 * The graph and labels are copied to the device and stay resident; labels
 * are compacted per partition and stored vertex-major (the n x k membership
 * matrix of the complexity analysis).  Errors: CC_ERR_INVALID,
 * CC_ERR_OVERFLOW, CC_ERR_OOM, CC_ERR_CUDA (then *out is NULL and nothing
 * leaks). */
cc_status cc_create(int32_t n, int64_t nnz, const int64_t* row_off, const int32_t* col, int32_t k,
                    const int32_t* labels, const cc_options* opt, cc_ctx** out);

/* As cc_create, with row_off, col and labels in device memory (same layouts).
 * stream: the cudaStream_t to use (NULL: the context creates its own).  The
 * device buffers are read on that stream before the call returns. */
cc_status cc_create_dev(int32_t n, int64_t nnz, const int64_t* row_off_dev, const int32_t* col_dev,
                        int32_t k, const int32_t* labels_dev, const cc_options* opt, void* stream,
                        cc_ctx** out);

/* One job of a batch: the arguments of cc_create for that job (host memory). */
typedef struct {
    int32_t n;
    int64_t nnz;
    const int64_t* row_off;
    const int32_t* col;
    int32_t k;
    const int32_t* labels;
} cc_job_desc;

/* Creates one context for `jobs` independent consensus jobs (the batched
 * form: many small problems solved together).  Each job follows the rules of
 * cc_create; the jobs are held on the device as one disjoint union (job j's
 * vertices follow those of jobs 0..j-1) and every sweep runs all of them in
 * the same kernel launches.  Each job keeps its own guard decisions,
 * objective, stopping condition and history, so its results are those of
 * running it alone in its own context.  A run stops when every job has
 * stopped (a job stops on a sweep with no proposal or at the sweep limit).
 * Per-job results: cc_job_objective, cc_job_history, cc_job_labels.
 * cc_consensus_labels / cc_cluster_ids / cc_set_cluster_ids work on all jobs
 * at once: int32[sum n_j], job after job, ids and labels local to each job.
 * cc_sweep (info must be NULL), cc_history, cc_objective and
 * cc_objective_recompute need a single-job context (else CC_ERR_INVALID).
 * Errors as cc_create; a message names the first job that failed. */
cc_status cc_batch_create(int32_t jobs, const cc_job_desc* descs, const cc_options* opt, cc_ctx** out);

/* Distances between a job's consensus and one of its input partitions P_i
 * (Methods, "Evaluation metrics"; the standard definitions):
 *   mirkin         Mirkin(C, P_i) over ordered pairs (pairs co-clustered in
 *                  exactly one of the two); sum_i mirkin = the job's F
 *   split_join     van Dongen's split-join distance: 2n - sum over clusters
 *                  c of max_l |c & l| - sum over classes l of P_i of max_c |c & l|
 *   rand_distance  Rand distance = mirkin / (n (n - 1)), 0 for n = 1
 *   vi             Meila's variation of information H(C|P_i) + H(P_i|C) in
 *                  nats, p(c, l) = |c & l| / n (fp64 sums; the order of the
 *                  sums is not fixed, so the last bits may vary)            */
typedef struct {
    int64_t mirkin;
    int64_t split_join;
    double rand_distance;
    double vi;
} cc_partition_metrics;

/* The distances of every job's current consensus to each of its input
 * partitions: out (caller-allocated, sum_j k_j entries) receives job 0's k_0
 * partitions in order, then job 1's, and so on.  Rebuilds the contingency
 * table at its current capacity first (the results of later sweeps do not
 * change).  Errors: CC_ERR_OOM (scratch), CC_ERR_CUDA. */
cc_status cc_metrics(cc_ctx* ctx, cc_partition_metrics* out);

/* Grouping homogeneous partitions (Methods, "Grouping homogeneous
 * partitions"): the distances between every pair of the job's input
 * partitions, out[a * k + i] = distances of P_a to P_i (k x k entries,
 * caller-allocated; the diagonal is zero).  Each P_a in turn is made the
 * consensus and measured as by cc_metrics; the context's consensus, objective
 * and history are restored afterwards.  Single-job contexts only.  Errors as
 * cc_metrics, CC_ERR_INVALID for a batch. */
cc_status cc_partition_distances(cc_ctx* ctx, cc_partition_metrics* out);

/* Groups k partitions: the complete graph over them, weighted by
 * distance[a * k + b] (e.g. the split_join field of cc_partition_distances),
 * keeps the edges whose weight is not above lambda; its connected components
 * are the groups.  group_of (int32[k], written) numbers them from 0 in order
 * of their first partition; *groups (may be NULL) receives their count.
 * Host only.  Errors: CC_ERR_INVALID. */
cc_status cc_group_partitions(int32_t k, const int64_t* distance, int64_t lambda, int32_t* group_of,
                              int32_t* groups);

/* Number of jobs of the context (1 for cc_create / cc_create_dev). */
cc_status cc_job_count(const cc_ctx* ctx, int32_t* out);

/* F of job `job` (ordered pairs, as cc_objective) and, if sweeps is not NULL,
 * the number of sweeps recorded for it since creation or the last reset. */
cc_status cc_job_objective(cc_ctx* ctx, int32_t job, int64_t* out, int32_t* sweeps);

/* The sweep records of job `job`, as cc_history.  A batch context keeps the
 * last max(64, max_sweeps option) records per job; a single-job one 65536. */
cc_status cc_job_history(cc_ctx* ctx, int32_t job, int32_t max, cc_sweep_info* out, int32_t* count);

/* The consensus of job `job` as int32[n_j] host, renumbered as by
 * cc_consensus_labels of that job alone. */
cc_status cc_job_labels(cc_ctx* ctx, int32_t job, int32_t* out);

/* The batch calls under the names of the interface's first description
 * (a batch context is a cc_ctx from cc_batch_create):
 * cc_batch_run  = cc_run_until_converged without the sweep count: the whole
 *                 run of every job (one graph launch for a batch context).
 * cc_batch_result = job `job`'s consensus labels (int32[n_j] host, as
 *                 cc_job_labels) and objective (as cc_job_objective); either
 *                 output may be NULL, not both.  Errors as those calls. */
cc_status cc_batch_run(cc_ctx* ctx, int32_t max_sweeps);
cc_status cc_batch_result(cc_ctx* ctx, int32_t job, int32_t* labels_out, int64_t* objective_out);

/* Uses the given cudaStream_t (NULL: the context's own) for later calls. */
cc_status cc_set_stream(cc_ctx* ctx, void* stream);

/* Returns the context to the singleton start (C[v] = v, F = F0) with the
 * inputs kept resident; the sweep history is cleared. */
cc_status cc_reset(cc_ctx* ctx);

/* Replaces the consensus with C (host int32[n], cluster ids in [0, n); any
 * ids, not only founding vertices) and rebuilds sizes, contingency counts and
 * F from it; the sweep history is kept.  This is a warm start (for instance
 * resuming from a saved consensus: the state of a run is C alone, everything
 * else is derived from C and the inputs).  The paper always starts from
 * singletons (The algorithm: Initialization); this call generalises that step.
 * Errors: CC_ERR_INVALID (an id outside [0, n)), CC_ERR_CUDA. */
cc_status cc_set_cluster_ids(cc_ctx* ctx, const int32_t* C);

/* Runs one synchronous sweep (Parallel algorithm section) and, if info is not
 * NULL, writes its record (info must be NULL for a batch).  A sweep with no
 * proposal changes nothing.
 * Errors: CC_ERR_TABLE_FULL, CC_ERR_CUDA, CC_ERR_INVALID (debug check). */
cc_status cc_sweep(cc_ctx* ctx, cc_sweep_info* info);

/* Runs sweeps until one has no proposal (the stopping condition of The
 * algorithm) or max_sweeps sweeps ran (max_sweeps <= 0: the option's limit).
 * Sweeps are submitted as CUDA graphs of up to 4 unrolled sweeps (a sweep is
 * skipped on the device once the run has stopped); the host reads the stop
 * flag after each graph, so a run costs one synchronisation per 4 sweeps.
 * A context of several jobs (cc_batch_create; unless no_regions is set) runs
 * instead as one graph launch: a conditional loop repeats the sweep until
 * the run stops, and the host synchronises once.
 * *sweeps_done (may be NULL) counts every sweep run, the final empty one
 * included.  Errors as cc_sweep. */
cc_status cc_run_until_converged(cc_ctx* ctx, int32_t max_sweeps, int32_t* sweeps_done);

/* Device time of each sweep of the last cc_run_until_converged / cc_sweep
 * call, from CUDA events recorded inside its graphs on the context's stream:
 * sweep_ms[s] covers sweep s (all its kernels), propose_ms[s] its proposal
 * kernels (k_own, k_edges, k_collect); with colour_batched, entry s covers
 * the s-th colour class run (a sweep is one run of every class).  A run that
 * was one graph launch (a context of several jobs) has one entry for it, with
 * propose_ms 0 (the proposal kernels are not timed apart inside the loop).  At most max entries are written to
 * each non-NULL array; *count receives the number of sweeps timed.  A sweep
 * abandoned for lack of table space and retried is timed once per attempt. */
cc_status cc_last_run_timing(cc_ctx* ctx, int32_t max, float* sweep_ms, float* propose_ms, int32_t* count);

/* Current state of the contingency hash (synchronises the stream). */
cc_status cc_table_stats(cc_ctx* ctx, cc_table_info* out);

/* Number of CUDA kernels the context has run since creation: every kernel it
 * launched directly, every kernel node of its sweep graphs that sits outside
 * a conditional region (whether or not a stopped sweep returned from it at
 * once), and the kernels of the conditional regions that ran (the heavy
 * path, the second attempt of its rebuild, its evaluation, its rollback, the
 * light path and the end-of-sweep rebuild of a sweep are IF nodes, entered
 * only when needed; their gates count them on the device).  Synchronises the
 * context's stream. */
cc_status cc_launch_count(const cc_ctx* ctx, int64_t* out);

/* Copies the records of the sweeps run since creation or the last reset,
 * oldest first: at most max entries into out, the total count into *count.
 * Single-job contexts only (batches: cc_job_history). */
cc_status cc_history(cc_ctx* ctx, int32_t max, cc_sweep_info* out, int32_t* count);

/* F(C) = sum_i Mirkin(C, P_i), ordered pairs (Eq. objective1), as kept
 * incrementally by the sweeps.  Single-job contexts only (cc_job_objective). */
cc_status cc_objective(cc_ctx* ctx, int64_t* out);

/* F(C) recomputed from scratch on the device from C and the labels
 * (k sum_c |c|^2 + sum_ij |P_ij|^2 - 2 sum_{c,i,j} n(c,i,j)^2), for checks.
 * Single-job contexts only. */
cc_status cc_objective_recompute(cc_ctx* ctx, int64_t* out);

/* The consensus as int32[n] (caller-allocated host buffer), clusters
 * renumbered 0..b-1 in order of first appearance by vertex index. */
cc_status cc_consensus_labels(cc_ctx* ctx, int32_t* out);

/* The raw cluster ids (founding vertices) as int32[n] host, for parity checks.
 * A batch gives int32[sum n_j], each job's ids local to the job. */
cc_status cc_cluster_ids(cc_ctx* ctx, int32_t* out);

/* Device pointer to the context's int32[n] cluster-id array (valid until the
 * next call that modifies the context or cc_destroy); for zero-copy readers.
 * In a batch the ids are those of the union: job j's ids are offset by the
 * number of vertices of jobs 0..j-1. */
cc_status cc_cluster_ids_dev(cc_ctx* ctx, const int32_t** out);

/* Message of the last failure on this context ("" if none).  Owned by the
 * context; valid until the next call on it.  A NULL ctx gives the message of
 * the last failed creation or context-free call in this thread. */
const char* cc_last_error(const cc_ctx* ctx);

/* Frees every resource of the context.  NULL is allowed. */
void cc_destroy(cc_ctx* ctx);

/* Device bytes a context for these jobs would hold (*persistent, until
 * cc_destroy) and at most during its creation (*peak), computed on the host
 * from n, nnz and k of each job and the options (the data pointers of the
 * descriptors are not read and may be NULL).  Either output may be NULL.
 * Errors: those of cc_batch_create's size and option checks. */
cc_status cc_estimate_bytes(int32_t jobs, const cc_job_desc* descs, const cc_options* opt, int64_t* persistent,
                            int64_t* peak);

/* Splits jobs into batches for cc_batch_create (host only; the data
 * pointers are not read): jobs are grouped by lane bin (the k ranges listed
 * under the served form below) and each group is cut, in job order, into
 * batches whose peak device bytes (cc_estimate_bytes) fit in budget_bytes
 * and that hold at most max_jobs jobs (max_jobs <= 0: no limit).
 * batch_of[j] (int32[jobs], written) receives job j's batch, numbered from 0
 * in order of lane bin, or -1 for a job that alone needs more than the
 * budget; *batches receives the number of batches.  Errors: CC_ERR_INVALID,
 * CC_ERR_OVERFLOW (a job's sizes, as in cc_create). */
cc_status cc_plan_batches(int32_t jobs, const cc_job_desc* descs, const cc_options* opt, int64_t budget_bytes,
                          int32_t max_jobs, int32_t* batch_of, int32_t* batches);

/* ---- served form: a request loop with continuous batching ---------------
 * A server takes consensus jobs as they arrive and keeps them resident on
 * the GPU while they run.  Waiting jobs are admitted in arrival order into
 * contexts of many jobs (as cc_batch_create) while a context slot is free and
 * the new context's device bytes (cc_estimate_bytes, peak) fit in what the
 * budget has left; the oldest waiting job opens a context and later ones of
 * the same lane bin (k in the same range: 1..10, 11..20, 21..40, 41..80,
 * 81..160, above 160) and of similar size (n within a factor 4 of the first
 * job's) join it while they fit.  Every context runs on its own stream, so
 * contexts admitted while others run overlap with them on the device;
 * streams of smaller contexts have higher CUDA priority.  Between two graph
 * launches of a context, every job of it whose run has stopped is released
 * at once (labels, objective, sweeps), whatever its siblings still do, and
 * a waiting job of the same lane bin that fits the released job's place (no
 * more vertices, CSR entries, partitions or label rows than it, and at least
 * a quarter of its vertices and CSR entries) is loaded
 * into that place and joins the running union from its singleton start
 * (not with colour_batched).  A job's results are those of running it
 * alone.  Single-threaded:
 * all calls on one server come from one thread at a time.  Device memory
 * comes from a memory pool of the server (stream-ordered allocation). */
typedef struct cc_server cc_server;

typedef struct {
    int64_t budget_bytes;   /* device bytes the server may hold for contexts; 0 = 80% of the
                               free device memory at creation */
    int32_t max_active;     /* contexts in flight at once (1..64); 0 = 8 */
    int32_t max_batch_jobs; /* jobs admitted into one context; 0 = 256 */
    int32_t reserved[4];    /* must be zero */
} cc_server_options;

typedef struct {
    int64_t submitted, admitted, completed, failed;
    int64_t batches;        /* contexts created */
    int64_t max_in_flight;  /* most contexts in flight at once */
    int64_t in_flight, queued;
    int64_t budget_bytes, bytes_in_use, peak_bytes;
    int64_t admitted_running; /* jobs loaded into the place of a finished job of a running context */
} cc_server_info;

/* Fills *o with the defaults above. */
void cc_server_default_options(cc_server_options* o);

/* Creates a server on the current device.  opt: options of every job
 * (max_sweeps is each job's sweep limit), or NULL for the defaults. */
cc_status cc_server_create(const cc_server_options* sopt, const cc_options* opt, cc_server** out);

/* Queues one job (host arrays as in cc_create) and returns at once with its
 * ticket.  Unlike the other calls, the job's arrays are borrowed until the
 * job is done: they must stay valid and unchanged until then.  labels_out
 * (int32[n], host) receives the job's consensus, renumbered as by
 * cc_consensus_labels.  Errors: the size checks of cc_create. */
cc_status cc_server_submit(cc_server* s, const cc_job_desc* job, int32_t* labels_out, int64_t* ticket);

/* Advances the server: harvests the contexts whose jobs have all stopped,
 * queues the next graph launch of those still running and admits waiting
 * jobs.  wait != 0: if nothing finished and nothing was admitted, keeps
 * polling (at most about a second) until something does.  Up to max_done
 * tickets of jobs done since the last report are written to done (*n_done
 * of them); *pending = jobs submitted and not yet done.  A job that fails
 * is done with a non-zero status (cc_server_job). */
cc_status cc_server_progress(cc_server* s, int32_t wait, int64_t* done, int32_t max_done, int32_t* n_done,
                             int64_t* pending);

/* State of a job: *done = 1 once its labels are written; its objective
 * (ordered pairs), sweeps run and cc_status.  Records are kept until
 * cc_server_destroy. */
cc_status cc_server_job(cc_server* s, int64_t ticket, int32_t* done, int64_t* F, int32_t* sweeps,
                        int32_t* status);

cc_status cc_server_stats(const cc_server* s, cc_server_info* out);

/* Message of the last failure on the server (NULL: of the last failed
 * cc_server_create in this thread). */
const char* cc_server_last_error(const cc_server* s);

/* Waits for the work in flight and frees everything.  NULL is allowed. */
void cc_server_destroy(cc_server* s);

/* ---- allocation-free output renumbering --------------------------------
 * The paper has no counterpart to this call; it serves callers of the
 * library.  It does what cc_consensus_labels does to a context's clusters,
 * but on caller-owned device buffers and without allocating any device
 * memory: no cudaMalloc, cudaFree or allocating library routine is called.
 * It is for code that cannot allocate at that point, e.g. code running under
 * a framework whose memory pool already holds the GPU's memory, or a
 * latency-bound path that must not pay for cudaMalloc / cudaFree (which can
 * synchronise the device).  Its temporary arrays live in one fixed array
 * compiled into the library: every GPU that loads libcc.so holds
 * CC_NOALLOC_SCRATCH_INTS ints (about 17 MB) of it until the process exits.
 *
 *   n           number of entries, 1 <= n <= CC_NOALLOC_MAX_N (else CC_ERR_INVALID)
 *   ids_dev     int32[n] device: cluster ids, each in [0, n) (else CC_ERR_INVALID),
 *               e.g. the array given by cc_cluster_ids_dev
 *   labels_dev  int32[n] device, written: ids renumbered 0..b-1 in order of
 *               first appearance by index
 *
 * The numbering runs over the n entries as one array.  For a single-job
 * context that is exactly cc_consensus_labels.  For a batch context,
 * cc_cluster_ids_dev holds union ids, and the result numbers the clusters
 * of all jobs together: job 0's labels, then job 1's labels plus the number
 * of clusters of job 0, and so on (each job's own labels, as cc_job_labels
 * gives them, are the result's slice for that job minus its first value).
 *   stream      cudaStream_t to run on (NULL: the legacy default stream); the
 *               call synchronises it before returning
 *
 * The first call on each device looks up the device address of the fixed
 * array (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The address is kept for the life of the
 * process: after a cudaDeviceReset of that device, do not call this entry
 * point again.  All calls on a device share the array, so calls
 * that overlap on the GPU (other streams, other host threads) race and give
 * wrong labels: serialise them.  Each call resets the part it needs, so
 * nothing carries over from the previous call.  Errors are reported through
 * cc_last_error(NULL). */
#define CC_NOALLOC_MAX_N (1 << 21)
#define CC_NOALLOC_SCRATCH_INTS (2 * CC_NOALLOC_MAX_N + CC_NOALLOC_MAX_N / 1024 + 64)
cc_status cc_renumber_noalloc(int32_t n, const int32_t* ids_dev, int32_t* labels_dev, void* stream);
/* The lane counts the autotuner (cc_options.autotune) chose on the current
 * device, per lane bin (0: 1..10 partitions, 1: 11..20, 2: 21..40, 3: 41..80,
 * 4: 81..160, 5: above): out[b] for b < bins (at most 6), 0 where no
 * context of that bin was tuned yet.  Never fails for a non-null out. */
cc_status cc_autotune_record(int32_t bins, int32_t* out);

/* CC_NOALLOC_MAX_N as compiled into the library (for bindings that cannot
 * read this header's macros).  Never fails. */
int32_t cc_noalloc_max_n(void);

#ifdef __cplusplus
}
#endif

#endif /* CC_H */
