// Allocation-free variant of the tile counting sort (pic_tile_sort_noalloc in gbpic.h).
//
// Some callers cannot let a library allocate device memory: an application that reserves its
// whole device budget in its own pool at start-up and forbids allocations afterwards, or code
// that runs where the CUDA allocator must not be entered.  This entry point sorts caller-owned
// arrays and takes its scratch (per-element ranks and the block sums of the scan) from a
// file-scope device array of fixed size instead of cudaMalloc.  The array exists once per GPU
// that loads the library and is held until the process exits.  Every call shares it and it
// keeps the previous call's contents: the kernels write every scratch word before reading it,
// and the histogram (the caller's key_start) is cleared at the start of each call.  Two calls
// whose work overlaps on the GPU (different streams, no ordering between them) race on the
// scratch and give wrong results.
#include "gbpic_internal.cuh"

#include <algorithm>
#include <mutex>

namespace gbpic {
namespace {

constexpr int kNaThreads = 1024;
constexpr int kNaSeg = 2 * kNaThreads;
constexpr int64_t kNaMaxN = PIC_NOALLOC_MAX_N;
constexpr int64_t kNaMaxKeys = PIC_NOALLOC_MAX_KEYS;
// ranks of up to kNaMaxN elements + scan block sums of up to kNaMaxKeys + 1 counters
constexpr int64_t kNaScanWords = (kNaMaxKeys + 1 + kNaSeg - 1) / kNaSeg + 64;
constexpr int64_t kNaWords = kNaMaxN + kNaScanWords;

static __device__ __align__(256) int g_noalloc_scratch[kNaWords];

struct NaKey {
    int T[3], nt[3], tile_cells, n[3], n_keys;
};

// key of a packed cell; cells outside the grid count as dummies (key n_keys)
__device__ __forceinline__ int na_key(int cell, const NaKey &t)
{
    const int i = cell & 1023, j = (cell >> 10) & 1023, k = cell >> 20;
    if (cell < 0 || i >= t.n[0] || j >= t.n[1] || k >= t.n[2]) return t.n_keys;
    const int tile = ((k / t.T[2]) * t.nt[1] + j / t.T[1]) * t.nt[0] + i / t.T[0];
    const int local = ((k % t.T[2]) * t.T[1] + j % t.T[1]) * t.T[0] + i % t.T[0];
    return tile * t.tile_cells + local;
}

__global__ void k_na_count(const int *cells, int n, NaKey t, int n_keys, int *hist, int *rank)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int cell = cells[p];
        const int key = na_key(cell, t);
        rank[p] = atomicAdd(hist + key, 1);
    }
}

__global__ void k_na_scatter(const int *cells, int n, NaKey t, const int *start, const int *rank, int *order)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int key = na_key(cells[p], t);
        if (key >= t.n_keys) continue;
        order[start[key] + rank[p]] = p;
    }
}

// exclusive scan of one kNaSeg segment per block; block totals to sums (when non-null)
__global__ void __launch_bounds__(kNaThreads) k_na_scan_blocks(int *data, long long n, int *sums)
{
    __shared__ int warp_tot[32];
    const long long i0 = (long long)blockIdx.x * kNaSeg + 2 * threadIdx.x;
    const int a = i0 < n ? data[i0] : 0;
    const int b = i0 + 1 < n ? data[i0 + 1] : 0;
    int v = a + b;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int w = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    const int incl = v + (wid > 0 ? warp_tot[wid - 1] : 0);
    const int excl = incl - (a + b);
    if (i0 < n) data[i0] = excl;
    if (i0 + 1 < n) data[i0 + 1] = excl + a;
    if (threadIdx.x == kNaThreads - 1 && sums) sums[blockIdx.x] = incl;
}

__global__ void k_na_scan_add(int *data, long long n, const int *offs)
{
    const int add = offs[blockIdx.x];
    const long long i0 = (long long)blockIdx.x * kNaSeg + threadIdx.x;
    if (i0 < n) data[i0] += add;
    if (i0 + kNaThreads < n) data[i0 + kNaThreads] += add;
}

cudaError_t na_scan(cudaStream_t st, int *data, long long n, int *scratch)
{
    const long long nb = (n + kNaSeg - 1) / kNaSeg;
    if (nb <= 1) {
        k_na_scan_blocks<<<1, kNaThreads, 0, st>>>(data, n, nullptr);
        return cudaGetLastError();
    }
    k_na_scan_blocks<<<(unsigned)nb, kNaThreads, 0, st>>>(data, n, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = na_scan(st, scratch, nb, scratch + nb)) != cudaSuccess) return e;
    k_na_scan_add<<<(unsigned)nb, kNaThreads, 0, st>>>(data, n, scratch);
    return cudaGetLastError();
}

// Device address of the scratch array, looked up once per device (with that device current).
std::mutex g_na_mu;
int *g_na_ptr[64] = {nullptr};

cudaError_t na_scratch(int dev, int **out)
{
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_na_ptr[dev] = static_cast<int *>(p);
    }
    *out = g_na_ptr[dev];
    return cudaSuccess;
}

}  // namespace

void set_global_error(const std::string &m);

int na_fail(int code, const std::string &m)
{
    set_global_error(m);
    return code;
}

}  // namespace gbpic

extern "C" int pic_tile_sort_noalloc(const int32_t *cells, int64_t n, const int grid[3], const int tile[3],
                                     int32_t *order, int32_t *key_start, void *stream)
{
    using namespace gbpic;
    if (!grid || !tile || (n > 0 && (!cells || !order)) || !key_start || n < 0)
        return na_fail(PIC_ERR_ARG, "pic_tile_sort_noalloc: null pointer or negative n");
    if (n > kNaMaxN)
        return na_fail(PIC_ERR_ARG, "pic_tile_sort_noalloc: n = " + std::to_string(n) + " exceeds the maximum " +
                                        std::to_string(kNaMaxN));
    NaKey t{};
    int64_t ntiles = 1;
    for (int d = 0; d < 3; d++) {
        const int lim = d == 2 ? 2048 : 1024;
        if (grid[d] < 1 || grid[d] > lim || tile[d] < 1 || tile[d] > grid[d])
            return na_fail(PIC_ERR_ARG, "pic_tile_sort_noalloc: grid or tile size out of range");
        t.T[d] = tile[d];
        t.n[d] = grid[d];
        t.nt[d] = (grid[d] + tile[d] - 1) / tile[d];
        ntiles *= t.nt[d];
    }
    // sizes in 64-bit: a tile as large as the grid's limits has more cells than an int holds
    const int64_t tile_cells = (int64_t)tile[0] * tile[1] * tile[2];
    const int64_t n_keys = ntiles * tile_cells;
    if (n_keys <= 0 || n_keys > kNaMaxKeys)
        return na_fail(PIC_ERR_ARG, "pic_tile_sort_noalloc: " + std::to_string(n_keys) + " keys exceed the maximum " +
                                        std::to_string(kNaMaxKeys));
    t.tile_cells = (int)tile_cells;
    t.n_keys = (int)n_keys;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return na_fail(PIC_ERR_CUDA, "pic_tile_sort_noalloc: no current device");
    int *scratch = nullptr;
    cudaError_t e = na_scratch(dev, &scratch);
    if (e != cudaSuccess) return na_fail(PIC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int *rank = scratch;
    int *scan_tmp = scratch + kNaMaxN;
    if ((e = cudaMemsetAsync(key_start, 0, sizeof(int32_t) * (n_keys + 1), st)) != cudaSuccess)
        return na_fail(PIC_ERR_CUDA, std::string("clear key_start: ") + cudaGetErrorString(e));
    if (n > 0) {
        k_na_count<<<592, 256, 0, st>>>(cells, (int)n, t, (int)n_keys, key_start, rank);
        if ((e = cudaGetLastError()) != cudaSuccess) return na_fail(PIC_ERR_CUDA, cudaGetErrorString(e));
    }
    if ((e = na_scan(st, key_start, n_keys + 1, scan_tmp)) != cudaSuccess)
        return na_fail(PIC_ERR_CUDA, cudaGetErrorString(e));
    if (n > 0) {
        k_na_scatter<<<592, 256, 0, st>>>(cells, (int)n, t, key_start, rank, order);
        if ((e = cudaGetLastError()) != cudaSuccess) return na_fail(PIC_ERR_CUDA, cudaGetErrorString(e));
    }
    return PIC_OK;
}
