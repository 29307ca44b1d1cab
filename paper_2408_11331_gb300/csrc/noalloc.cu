// cc_renumber_noalloc: the output renumbering of cc_consensus_labels for
// callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not an option, for example
// inside a framework whose caching allocator has already reserved the GPU's
// memory (a cudaMalloc there fails or fights the pool), or on a latency-bound
// path that must not pay for cudaMalloc / cudaFree, which can synchronise the
// whole device.  Such callers own their input and output buffers; the
// temporary arrays the renumbering needs live in a fixed array compiled into
// the library instead of being allocated per call.
//
// The scratch array is one file-scope __device__ array, so every GPU that
// loads the library holds CC_NOALLOC_SCRATCH_INTS ints (about 17 MB) until the
// process exits, and every call on a device shares it.
#include <mutex>
#include <string>

#include "cc_internal.cuh"

// first[n] + rank[n] + per-block counts + one error flag
static __device__ __align__(256) int g_noalloc_scratch[CC_NOALLOC_SCRATCH_INTS];

namespace ccg {

namespace {

std::mutex g_setup_mutex;
int* g_scratch_addr[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

// Host-side address of the scratch array on the current device, looked up
// once per device (the symbol's name is only a stand-in on the host).
cudaError_t scratch_address(int** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<int*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// Scratch layout for a call with n ids: first[0..n), rank[n..2n),
// block counts [2n .. 2n+nb), error flag at the last int of the array.
__global__ void k_na_reset(int n, int* first, int* flag)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) first[c] = 0x7fffffff;
    if (blockIdx.x == 0 && threadIdx.x == 0) *flag = 0;
}

__global__ void k_na_first(int n, const int* __restrict__ ids, int* first, int* flag)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int c = ids[v];
        if (c < 0 || c >= n) *flag = 1;
        else atomicMin(&first[c], (int)v);
    }
}

// rank[v] = 1 if v is the least vertex of its cluster; counts per block of 1024.
__global__ void __launch_bounds__(1024) k_na_marks(int n, const int* __restrict__ ids, const int* __restrict__ first,
                                                   int* rank, int* counts, const int* flag)
{
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int f = 0;
    if (v < n && *flag == 0) f = first[ids[v]] == v;
    if (v < n) rank[v] = f;
    if (f) atomicAdd(&cnt, 1);
    __syncthreads();
    if (threadIdx.x == 0) counts[blockIdx.x] = cnt;
}

// Exclusive scan of the nb block counts by one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_na_scan_counts(int nb, int* counts)
{
    __shared__ int part[1024];
    const int per = (nb + 1023) / 1024;
    const int lo = threadIdx.x * per, hi = min(nb, lo + per);
    int sum = 0;
    for (int b = lo; b < hi; ++b) sum += counts[b];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int y = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += y;
        __syncthreads();
    }
    int run = part[threadIdx.x] - sum;
    for (int b = lo; b < hi; ++b) {
        const int x = counts[b];
        counts[b] = run;
        run += x;
    }
}

// rank[v] becomes the number of cluster heads before v (exclusive scan).
__global__ void __launch_bounds__(1024) k_na_rank(int n, int* rank, const int* counts)
{
    __shared__ int buf[1024];
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int f = v < n ? rank[v] : 0;
    buf[threadIdx.x] = f;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int y = threadIdx.x >= (unsigned)o ? buf[threadIdx.x - o] : 0;
        __syncthreads();
        buf[threadIdx.x] += y;
        __syncthreads();
    }
    if (v < n) rank[v] = counts[blockIdx.x] + buf[threadIdx.x] - f;
}

__global__ void k_na_relabel(int n, const int* __restrict__ ids, const int* __restrict__ first,
                             const int* __restrict__ rank, int* out, const int* flag)
{
    if (*flag) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) out[v] = rank[first[ids[v]]];
}

}  // namespace

}  // namespace ccg

extern "C" int32_t cc_noalloc_max_n(void)
{
    return CC_NOALLOC_MAX_N;
}

extern "C" cc_status cc_renumber_noalloc(int32_t n, const int32_t* ids_dev, int32_t* labels_dev, void* stream)
{
    using namespace ccg;
    if (n < 1 || n > CC_NOALLOC_MAX_N) {
        set_thread_error("cc_renumber_noalloc: n must lie in [1, " + std::to_string(CC_NOALLOC_MAX_N) +
                         "], the size of its built-in scratch");
        return CC_ERR_INVALID;
    }
    if (!ids_dev || !labels_dev) {
        set_thread_error("cc_renumber_noalloc: null pointer");
        return CC_ERR_INVALID;
    }
    int* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        set_thread_error(std::string("cc_renumber_noalloc: scratch address: ") + cudaGetErrorString(e));
        return CC_ERR_CUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nb = (n + 1023) / 1024;
    int* first = scratch;
    int* rank = scratch + n;
    int* counts = scratch + 2 * (size_t)n;
    int* flag = scratch + (CC_NOALLOC_SCRATCH_INTS - 1);
    const int g = nb < 1024 ? nb : 1024;
    k_na_reset<<<g, 1024, 0, s>>>(n, first, flag);
    k_na_first<<<g, 1024, 0, s>>>(n, ids_dev, first, flag);
    k_na_marks<<<nb, 1024, 0, s>>>(n, ids_dev, first, rank, counts, flag);
    k_na_scan_counts<<<1, 1024, 0, s>>>(nb, counts);
    k_na_rank<<<nb, 1024, 0, s>>>(n, rank, counts);
    k_na_relabel<<<g, 1024, 0, s>>>(n, ids_dev, first, rank, labels_dev, flag);
    e = cudaGetLastError();
    int bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_thread_error(std::string("cc_renumber_noalloc: ") + cudaGetErrorString(e));
        return CC_ERR_CUDA;
    }
    if (bad) {
        set_thread_error("cc_renumber_noalloc: cluster ids must lie in [0, n)");
        return CC_ERR_INVALID;
    }
    return CC_OK;
}
