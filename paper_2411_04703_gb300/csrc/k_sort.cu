// Counting sort of a species by tile-major cell key (locality for the particle kernel) and
// construction of its (tile, chunk) work items.  Dummy particles get the extra key n_keys and
// are dropped (compaction).  Histogram with global atomics -> exclusive scan of the tile totals
// -> exclusive scan of the keys of the tiles that hold particles -> scatter.  A bunch in a large
// grid fills few tiles, so the key counters of the others are never touched.  The order among
// particles of one cell is not fixed (atomic ranks).
#include "gbpic_internal.cuh"

namespace gbpic {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanSeg = 2 * kScanThreads;

// Sort key of a particle: tiles in x-fastest order; inside a tile the cells in (x fastest, z,
// y) order; inside a cell the octant of the offset (bit d set when offset_d >= 1/2).  A warp's
// 32 consecutive cells then form an 8 x 4 (x, z) block at one y, and the particles of a cold
// lattice come in the same octant order in every cell.
__device__ __forceinline__ int tile_key(const float4 &P, const TileDev &t)
{
    const int cell = __float_as_int(P.w);
    const int i = t.cc.i(cell), j = t.cc.j(cell), k = t.cc.k(cell);
    const int tile = ((k / t.T[2]) * t.nt[1] + j / t.T[1]) * t.nt[0] + i / t.T[0];
    const int local = ((j % t.T[1]) * t.T[2] + k % t.T[2]) * t.T[0] + i % t.T[0];
    const int oct = (P.x >= 0.5f) | ((P.y >= 0.5f) << 1) | ((P.z >= 0.5f) << 2);
    return (tile * t.tile_cells + local) * 8 + oct;
}

// Key counters (the rank of each particle among its key) and particles per tile.  The lanes of a
// warp mostly share a tile (the particles were sorted by tile last time), so a tile's counter
// takes one atomic per warp.
__global__ void k_sort_count(SpeciesDev sp, TileDev t, int n_keys, int *hist, int *rank, int *tile_cnt)
{
    const int n = sp.count[0];
    const int kpt = t.tile_cells * 8;
    const int lane = threadIdx.x & 31;
    for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const int p = base + threadIdx.x;
        int tile = -1 - lane;                      // no tile: a value no other lane has
        if (p < n) {
            const float4 P = sp.pos[p];
            const bool live = __float_as_int(P.w) >= 0;
            const int key = live ? tile_key(P, t) : n_keys;
            rank[p] = atomicAdd(hist + key, 1);
            if (live) tile = key / kpt;
        }
        // the lanes in lane 0's tile add with one atomic, the others (rare) each with their own
        const int t0 = __shfl_sync(0xffffffffu, tile, 0);
        const unsigned m = __ballot_sync(0xffffffffu, tile == t0);
        if (tile >= 0) {
            if (tile != t0) atomicAdd(tile_cnt + tile, 1);
            else if (lane == 0) atomicAdd(tile_cnt + tile, __popc(m));
        }
    }
}

// Zero the key counters of the tiles that held particles at the last sort (every other counter
// is zero already), and the dummies' counter.
__global__ void k_zero_occupied(int *hist, const int *occ, int ntiles, int kpt, int n_keys)
{
    const long long tot = (long long)occ[ntiles] * kpt;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const long long e = i / kpt;
        hist[(long long)occ[e] * kpt + (i - e * kpt)] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) hist[n_keys] = 0;
}

// List the tiles holding particles (order free).
__global__ void k_occ_list(const int *tile_start, int ntiles, int *occ)
{
    const int tl = blockIdx.x * blockDim.x + threadIdx.x;
    if (tl < ntiles && tile_start[tl + 1] > tile_start[tl]) occ[atomicAdd(occ + ntiles, 1)] = tl;
}

// Exclusive scan of the key counters of each listed tile, offset by the tile's first slot: the
// key counters of empty tiles are neither read nor written.  One block per tile at a time; the
// keys pass through shared memory in segments of kTileSeg (coalesced in global memory, padded
// by one word per 16 so that each thread's run of 16 sits in distinct banks), with a carry from
// segment to segment.
constexpr int kTileScanThreads = 256;
constexpr int kTileRun = 16;
constexpr int kTileSeg = kTileScanThreads * kTileRun;
__global__ void __launch_bounds__(kTileScanThreads) k_tile_scan(int *hist, const int *tile_start, const int *occ,
                                                               int ntiles, int kpt)
{
    __shared__ int seg[kTileSeg + kTileSeg / kTileRun];
    __shared__ int warp_off[kTileScanThreads / 32];
    __shared__ int carry;
    const int n_occ = occ[ntiles];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int nw = kTileScanThreads / 32;
    for (int e = blockIdx.x; e < n_occ; e += gridDim.x) {
        const int tile = occ[e];
        int *keys = hist + (long long)tile * kpt;
        if (threadIdx.x == 0) carry = tile_start[tile];
        for (int s0 = 0; s0 < kpt; s0 += kTileSeg) {
            const int len = min(kTileSeg, kpt - s0);
            for (int k = threadIdx.x; k < kTileSeg; k += kTileScanThreads)
                seg[k + k / kTileRun] = k < len ? keys[s0 + k] : 0;
            __syncthreads();
            int *run = seg + threadIdx.x * (kTileRun + 1);
            int sum = 0;
#pragma unroll
            for (int i = 0; i < kTileRun; i++) sum += run[i];
            int incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane == 31) warp_off[w] = incl;
            __syncthreads();
            if (w == 0) {
                const int tot = lane < nw ? warp_off[lane] : 0;
                int wi = tot;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, wi, o);
                    if (lane >= o) wi += v;
                }
                if (lane < nw) warp_off[lane] = wi - tot;
            }
            __syncthreads();
            int x = carry + warp_off[w] + incl - sum;
#pragma unroll
            for (int i = 0; i < kTileRun; i++) {
                const int v = run[i];
                run[i] = x;
                x += v;
            }
            __syncthreads();
            for (int k = threadIdx.x; k < len; k += kTileScanThreads) keys[s0 + k] = seg[k + k / kTileRun];
            if (threadIdx.x == kTileScanThreads - 1) carry = x;   // the segment's end
            __syncthreads();
        }
    }
}

__global__ void k_sort_scatter(SpeciesDev sp, TileDev t, int n_keys, const int *start, const int *rank,
                               float4 *pos2, float4 *mom2, int *id2)
{
    const int n = sp.count[0];
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const float4 P = sp.pos[p];
        const int cell = __float_as_int(P.w);
        if (cell < 0) continue;
        const int dst = start[tile_key(P, t)] + rank[p];
        pos2[dst] = P;
        mom2[dst] = sp.mom[p];
        id2[dst] = sp.id[p];
    }
}

// Work of a tile: chunks of kChunk particles for the shared-memory path, or, for a tile with
// fewer than kSparse particles, one entry in the sparse list (global-memory path, a warp each).
__global__ void k_tile_chunks(const int *tile_start, int ntiles, int chunk, int *chunk_count, int *sparse_flag)
{
    const int tl = blockIdx.x * blockDim.x + threadIdx.x;
    if (tl > ntiles) return;
    if (tl == ntiles) {
        chunk_count[tl] = 0;
        sparse_flag[tl] = 0;
        return;
    }
    const int cnt = tile_start[tl + 1] - tile_start[tl];
    const bool sparse = cnt > 0 && cnt < kSparse;
    chunk_count[tl] = sparse ? 0 : (cnt + chunk - 1) / chunk;
    sparse_flag[tl] = sparse ? 1 : 0;
}

__global__ void k_fill_items(const int *chunk_start, const int *sparse_start, int ntiles, int2 *items,
                             int *sparse_tiles, int *count, const int *tile_start)
{
    const int tl = blockIdx.x * blockDim.x + threadIdx.x;
    if (tl < ntiles) {
        const int b = chunk_start[tl], e = chunk_start[tl + 1];
        for (int c = b; c < e; c++) items[c] = make_int2(tl, c - b);
        if (sparse_start[tl + 1] > sparse_start[tl]) sparse_tiles[sparse_start[tl]] = tl;
    }
    if (tl == 0) {
        count[0] = tile_start[ntiles];
        count[1] = tile_start[ntiles];
        count[2] = chunk_start[ntiles];
        count[3] = sparse_start[ntiles];
    }
}

// Block-wide exclusive scan of kScanSeg ints per block; the block total goes to sums.
__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(int *data, long long n, int *sums)
{
    __shared__ int warp_tot[32];
    const long long i0 = (long long)blockIdx.x * kScanSeg + 2 * threadIdx.x;
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
        warp_tot[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    const int incl = v + (wid > 0 ? warp_tot[wid - 1] : 0);
    const int excl = incl - (a + b);
    if (i0 < n) data[i0] = excl;
    if (i0 + 1 < n) data[i0 + 1] = excl + a;
    if (threadIdx.x == kScanThreads - 1 && sums) sums[blockIdx.x] = incl;
}

__global__ void k_scan_add(int *data, long long n, const int *offs)
{
    const int add = offs[blockIdx.x];
    const long long i0 = (long long)blockIdx.x * kScanSeg + threadIdx.x;
    if (i0 < n) data[i0] += add;
    if (i0 + kScanThreads < n) data[i0 + kScanThreads] += add;
}

cudaError_t scan_rec(cudaStream_t st, int *data, long long n, int *scratch, int64_t &kernels)
{
    const long long nb = (n + kScanSeg - 1) / kScanSeg;
    if (nb <= 1) {
        k_scan_blocks<<<1, kScanThreads, 0, st>>>(data, n, nullptr);
        kernels++;
        return cudaGetLastError();
    }
    k_scan_blocks<<<(unsigned)nb, kScanThreads, 0, st>>>(data, n, scratch);
    kernels++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = scan_rec(st, scratch, nb, scratch + nb, kernels);
    if (e != cudaSuccess) return e;
    k_scan_add<<<(unsigned)nb, kScanThreads, 0, st>>>(data, n, scratch);
    kernels++;
    return cudaGetLastError();
}

}  // namespace

// Scratch ints needed by exclusive_scan for n elements.
int64_t scan_scratch_size(int64_t n)
{
    int64_t tot = 0;
    while (n > kScanSeg) {
        n = (n + kScanSeg - 1) / kScanSeg;
        tot += n;
    }
    return tot + 16;
}

cudaError_t exclusive_scan(pic_ctx *c, int *data, int64_t n)
{
    if (scan_scratch_size(n) > c->hist_tmp_n) return cudaErrorInvalidValue;
    return scan_rec(c->stream, data, n, c->hist_tmp, c->kernels);
}

cudaError_t launch_sort(pic_ctx *c, int si)
{
    Species &s = c->sp[si];
    // work items small enough that a small species still gives every SM one (each item stages a
    // whole tile region, so items are kept as large as that allows)
    s.chunk = kChunk;
    while (s.chunk > kChunkMin && s.bound / s.chunk < (int64_t)c->num_sms) s.chunk /= 2;
    TileDev t = tile_dev(c, s);
    SpeciesDev sd = species_dev(c, s);
    const int n_keys = (int)c->n_keys;
    const int kpt = t.tile_cells * 8;
    const int grid = c->num_sms * 8;
    // the key counters are zero outside the tiles listed at the last sort: zero those, count,
    // scan the tile totals, then the keys of the tiles that hold particles now
    k_zero_occupied<<<grid, 256, 0, c->stream>>>(s.cell_start, s.occ, c->ntiles, kpt, n_keys);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(s.occ + c->ntiles, 0, sizeof(int), c->stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(s.tile_start, 0, sizeof(int) * (c->ntiles + 1), c->stream)) != cudaSuccess) return e;
    k_sort_count<<<grid, 256, 0, c->stream>>>(sd, t, n_keys, s.cell_start, s.rank, s.tile_start);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = exclusive_scan(c, s.tile_start, c->ntiles + 1)) != cudaSuccess) return e;
    k_occ_list<<<(c->ntiles + 255) / 256, 256, 0, c->stream>>>(s.tile_start, c->ntiles, s.occ);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_tile_scan<<<c->num_sms * 4, kTileScanThreads, 0, c->stream>>>(s.cell_start, s.tile_start, s.occ, c->ntiles, kpt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_sort_scatter<<<grid, 256, 0, c->stream>>>(sd, t, n_keys, s.cell_start, s.rank, s.pos2, s.mom2, s.id2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_tile_chunks<<<(c->ntiles + 1 + 255) / 256, 256, 0, c->stream>>>(s.tile_start, c->ntiles, s.chunk, s.chunk_start,
                                                                       s.sparse_start);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = exclusive_scan(c, s.chunk_start, c->ntiles + 1)) != cudaSuccess) return e;
    if ((e = exclusive_scan(c, s.sparse_start, c->ntiles + 1)) != cudaSuccess) return e;
    k_fill_items<<<(c->ntiles + 255) / 256, 256, 0, c->stream>>>(s.chunk_start, s.sparse_start, c->ntiles, s.items,
                                                                  s.sparse_tiles, s.count, s.tile_start);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    c->kernels += 7;   // zero, count, occupied list, tile scan, scatter, tile_chunks, fill_items
    std::swap(s.pos, s.pos2);
    std::swap(s.mom, s.mom2);
    std::swap(s.id, s.id2);
    return cudaSuccess;
}

}  // namespace gbpic
