// Partition distances between each job's consensus and its input partitions
// (Methods, "Evaluation metrics": Rand / Mirkin distance, split-join
// distance, variation of information), as reductions over the contingency
// table of the consensus.  The host turns the sums into the distances:
//   Mirkin_i  = sum_c |c|^2 + sum_l |P_il|^2 - 2 sum_{c,l} n(c,i,l)^2   (ordered pairs)
//   SJ_i      = 2n - sum_c max_l n(c,i,l) - sum_l max_c n(c,i,l)
//   VI_i      = (sum_c |c| log|c| + sum_l |P_il| log|P_il| - 2 sum n log n) / n
// (the variation of information H(C|P_i) + H(P_i|C) with p = n(c,i,l) / n).
#include <cmath>

#include "cc_internal.cuh"

namespace ccg {

namespace {

constexpr int kMetBlock = 256;

// Grid for grid-stride kernels: at most 8 resident blocks per SM of the current device.
inline int met_grid(long long work)
{
    const long long max_blocks = 8LL * device_sm_count();
    long long b = (work + kMetBlock - 1) / kMetBlock;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

// Largest index i with key[i] <= x among key[0..count).
__device__ __forceinline__ int job_by_start(const long long* key, int count, long long x)
{
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (key[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Per-partition sums go through shared memory when the context has at most
// kSmemParts partitions (one add per block and partition to global memory).
constexpr int kSmemParts = 1024;

// Table slots: sum n^2 and sum n log n per partition, max over clusters per label.
__global__ void k_met_table(SweepArgs a, MetricsArgs m, int parts)
{
    extern __shared__ unsigned char smem[];
    const bool shared = parts <= kSmemParts;
    long long* ssq = reinterpret_cast<long long*>(smem);
    double* sslog = reinterpret_cast<double*>(smem + sizeof(long long) * (shared ? parts : 0));
    if (shared) {
        for (int P = threadIdx.x; P < parts; P += blockDim.x) {
            ssq[P] = 0;
            sslog[P] = 0.0;
        }
        __syncthreads();
    }
    long long* sq = shared ? ssq : m.sq;
    double* slog = shared ? sslog : m.slog;
    const unsigned long long cap = a.st->mask + 1;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; s < cap; s += stride) {
        const ulonglong2 e = reinterpret_cast<const ulonglong2*>(a.table)[s];
        const int cnt = (int)(unsigned)(e.y & 0xffffffffull);
        if (e.x == kEmpty || cnt <= 0) continue;
        const int x = (int)(e.x >> 32), g = (int)(unsigned)(e.x & 0xffffffffull);
        const int j = a.jid[x];
        const int P = m.pfirst[j] + (g >> a.job[j].lshift);
        const long long c = cnt;
        atomicAdd(reinterpret_cast<unsigned long long*>(sq + P), (unsigned long long)(c * c));
        atomicAdd(slog + P, (double)c * log((double)c));
        atomicMax(m.lmax + m.lbase[j] + g, cnt);
    }
    if (shared) {
        __syncthreads();
        for (int P = threadIdx.x; P < parts; P += blockDim.x) {
            if (ssq[P]) atomicAdd(reinterpret_cast<unsigned long long*>(m.sq + P), (unsigned long long)ssq[P]);
            if (sslog[P] != 0.0) atomicAdd(m.slog + P, sslog[P]);
        }
    }
}

// Clusters: |c|^2 and |c| log |c| per job, and the largest overlap of each
// (cluster, partition) -- the count of the summary row's label, exact after
// a rebuild.
__global__ void k_met_clusters(SweepArgs a, MetricsArgs m, int parts)
{
    extern __shared__ unsigned char smem[];
    const bool shared = parts <= kSmemParts;
    long long* ssjc = reinterpret_cast<long long*>(smem);
    if (shared) {
        for (int P = threadIdx.x; P < parts; P += blockDim.x) ssjc[P] = 0;
        __syncthreads();
    }
    long long* sjc = shared ? ssjc : m.sjc;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < a.n; x += stride) {
        const long long s = a.size[x];
        if (s <= 0) continue;
        const int j = a.jid[x];
        const JobInfo& J = a.job[j];
        atomicAdd(reinterpret_cast<unsigned long long*>(m.csq + j), (unsigned long long)(s * s));
        atomicAdd(m.cslog + j, (double)s * log((double)s));
        const int4* S = a.summ + row_of(J, x);
        const int P0 = m.pfirst[j];
        for (int i = 0; i < J.k; ++i)
            atomicAdd(reinterpret_cast<unsigned long long*>(sjc + P0 + i), (unsigned long long)S[i].y);
    }
    if (shared) {
        __syncthreads();
        for (int P = threadIdx.x; P < parts; P += blockDim.x)
            if (ssjc[P]) atomicAdd(reinterpret_cast<unsigned long long*>(m.sjc + P), (unsigned long long)ssjc[P]);
    }
}

// Label classes: the largest overlap of each class with a cluster.
__global__ void k_met_labels(SweepArgs a, MetricsArgs m)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < m.nlabels; t += stride) {
        const int best = m.lmax[t];
        if (best <= 0) continue;
        const int j = job_by_start(m.lbase, a.jobs, t);
        const int P = m.pfirst[j] + (int)((t - m.lbase[j]) >> a.job[j].lshift);
        atomicAdd(reinterpret_cast<unsigned long long*>(m.sjl + P), (unsigned long long)best);
    }
}

// C := input partition i of job j as a consensus: every vertex in the cluster
// named by the least vertex of its class (the representative in its label id).
__global__ void k_ids_from_partition(SweepArgs a, int j, int i)
{
    const JobInfo J = a.job[j];
    const int mask = (1 << J.lshift) - 1;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = J.vo + (long long)blockIdx.x * blockDim.x + threadIdx.x; v < J.vo + J.n; v += stride)
        a.C[v] = (int)(J.vo + (a.G[row_of(J, v) + i] & mask));
}

}  // namespace

cudaError_t launch_ids_from_partition(const SweepArgs& a, long long n, int j, int i, cudaStream_t s)
{
    k_ids_from_partition<<<met_grid(n), kMetBlock, 0, s>>>(a, j, i);
    return cudaGetLastError();
}

cudaError_t launch_metrics(const SweepArgs& a, const MetricsArgs& m, int parts, cudaStream_t s)
{
    const size_t sm = parts <= kSmemParts ? (size_t)parts * 16 : 0;
    const size_t sm1 = parts <= kSmemParts ? (size_t)parts * 8 : 0;
    k_met_table<<<met_grid((long long)a.mask_max + 1), kMetBlock, sm, s>>>(a, m, parts);
    k_met_clusters<<<met_grid(a.n), kMetBlock, sm1, s>>>(a, m, parts);
    k_met_labels<<<met_grid(m.nlabels), kMetBlock, 0, s>>>(a, m);
    return cudaGetLastError();
}

}  // namespace ccg
