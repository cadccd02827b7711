// Coherent processing order for the trace: a counting sort of the photon
// indices by (chunk of 2^20 photons of the input order, cell of the origin in
// a 128 x 128 grid over the origins' x-y bounding box).  Rays of one warp
// then start close together (and, within a chunk of the caller's order,
// usually share a direction), so they walk the same BVH nodes and hit the
// same surfaces and the warp's lanes diverge far less.  A chunk's inputs
// (28 MB in FP32) stay in L2 while the trace reads them in cell order, so the
// reordered loads cost little DRAM traffic.  Results do not depend on the
// order: every photon keeps its index, its random stream and its output slot.
//
// Chunk size and grid were swept on the dish workload (chunks 2^17..2^23,
// grids 64..1024 cells per axis): 2^20 photons per chunk was fastest (the
// trace's DRAM reads fall from 24 GB to 2 GB per 5e7 photons against 2^22),
// and grids of 128..512 cells per axis traced within 1% of each other.
//
// The sort is one pass of a block-local counting sort: every block of
// 2^ORD_TILE_BITS photons (one tile of a chunk) counts its photons per cell
// in shared memory and writes them contiguously, [chunk][tile][cell]; one
// thread per (chunk, cell) turns its column into running offsets over the
// tiles (in place) and its total; the totals are scanned; a second pass places
// each photon at base(chunk, cell) + offset(tile, cell) + its rank in the
// block (shared-memory atomics only).  Every pass reads and writes coalesced.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "launch.h"

namespace robast {

constexpr int ORD_G = 128;                // grid cells per axis
constexpr int ORD_CELLS = ORD_G * ORD_G;  // 16384 cells: 64 KB of counters per block
constexpr int ORD_CHUNK_BITS = 20;        // chunks of 2^20 photons keep the caller's order
constexpr int ORD_TILE_BITS = 16;         // photons per block
constexpr int ORD_TILES_PER_CHUNK = 1 << (ORD_CHUNK_BITS - ORD_TILE_BITS);
constexpr int ORD_BLOCK = 1024;

__device__ __forceinline__ int ordered_int(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float unordered_float(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void ord_init(int* box) {
    if (threadIdx.x == 0) {
        box[0] = 0x7fffffff;
        box[1] = (int)0x80000000;
        box[2] = 0x7fffffff;
        box[3] = (int)0x80000000;
    }
}

template <typename T>
__global__ void ord_bounds(const T* o, long long n, int* box) {
    float lo0 = 3.4e38f, lo1 = 3.4e38f, hi0 = -3.4e38f, hi1 = -3.4e38f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float x = (float)o[i], y = (float)o[n + i];
        lo0 = fminf(lo0, x);
        hi0 = fmaxf(hi0, x);
        lo1 = fminf(lo1, y);
        hi1 = fmaxf(hi1, y);
    }
    for (int off = 16; off > 0; off >>= 1) {
        lo0 = fminf(lo0, __shfl_xor_sync(0xffffffffu, lo0, off));
        hi0 = fmaxf(hi0, __shfl_xor_sync(0xffffffffu, hi0, off));
        lo1 = fminf(lo1, __shfl_xor_sync(0xffffffffu, lo1, off));
        hi1 = fmaxf(hi1, __shfl_xor_sync(0xffffffffu, hi1, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(box + 0, ordered_int(lo0));
        atomicMax(box + 1, ordered_int(hi0));
        atomicMin(box + 2, ordered_int(lo1));
        atomicMax(box + 3, ordered_int(hi1));
    }
}

struct OrdMap {
    float x0, sx, y0, sy;  // cell = (coordinate - origin) * scale
};

__device__ __forceinline__ OrdMap ord_map(const int* box) {
    const float x0 = unordered_float(box[0]), x1 = unordered_float(box[1]);
    const float y0 = unordered_float(box[2]), y1 = unordered_float(box[3]);
    return OrdMap{x0, x1 > x0 ? (float)ORD_G / (x1 - x0) : 0.0f, y0, y1 > y0 ? (float)ORD_G / (y1 - y0) : 0.0f};
}

// cell of photon i; serpentine rows keep consecutive cells adjacent
template <typename T>
__device__ __forceinline__ int ord_cell(const T* o, long long n, long long i, const OrdMap& m) {
    int cx = (int)(((float)o[i] - m.x0) * m.sx), cy = (int)(((float)o[n + i] - m.y0) * m.sy);
    cx = cx < 0 ? 0 : (cx >= ORD_G ? ORD_G - 1 : cx);
    cy = cy < 0 ? 0 : (cy >= ORD_G ? ORD_G - 1 : cy);
    return cy * ORD_G + ((cy & 1) ? ORD_G - 1 - cx : cx);
}

// Pass 1: per-block cell counts, to counts[(chunk * TILES + tile) * CELLS + cell] (the
// block's tile index is blockIdx.x).  Blocks past n (in the last chunk) write zeros.
template <typename T>
__global__ void __launch_bounds__(ORD_BLOCK) ord_count(const T* o, long long n, const int* box, unsigned* counts) {
    extern __shared__ unsigned h[];
    for (int c = threadIdx.x; c < ORD_CELLS; c += ORD_BLOCK) h[c] = 0;
    __syncthreads();
    const OrdMap m = ord_map(box);
    const long long b0 = (long long)blockIdx.x << ORD_TILE_BITS;
    const long long b1 = min(n, b0 + (1LL << ORD_TILE_BITS));
    for (long long i = b0 + threadIdx.x; i < b1; i += ORD_BLOCK) atomicAdd(&h[ord_cell(o, n, i, m)], 1u);
    __syncthreads();
    unsigned* dst = counts + (long long)blockIdx.x * ORD_CELLS;
    for (int c = threadIdx.x; c < ORD_CELLS; c += ORD_BLOCK) dst[c] = h[c];
}

// Per (chunk, cell): the column of tile counts becomes running offsets (exclusive, in
// place) and the column total goes to totals[chunk * CELLS + cell].
__global__ void ord_columns(unsigned* counts, long long nchunks, unsigned* totals) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;  // chunk * CELLS + cell
    if (k >= nchunks * ORD_CELLS) return;
    const long long chunk = k / ORD_CELLS, cell = k % ORD_CELLS;
    unsigned* col = counts + chunk * ORD_TILES_PER_CHUNK * (long long)ORD_CELLS + cell;
    unsigned run = 0;
    for (int t = 0; t < ORD_TILES_PER_CHUNK; ++t) {
        const unsigned v = col[(long long)t * ORD_CELLS];
        col[(long long)t * ORD_CELLS] = run;
        run += v;
    }
    totals[k] = run;
}

// Pass 2: each photon at base(chunk, cell) + offset(tile, cell) + its rank in the block.
template <typename T>
__global__ void __launch_bounds__(ORD_BLOCK) ord_place(const T* o, long long n, const int* box, const unsigned* offs,
                                                      const unsigned* base, int* order) {
    extern __shared__ unsigned h[];
    const long long chunk = blockIdx.x / ORD_TILES_PER_CHUNK;
    const unsigned* src = offs + (long long)blockIdx.x * ORD_CELLS;
    const unsigned* bc = base + chunk * ORD_CELLS;
    for (int c = threadIdx.x; c < ORD_CELLS; c += ORD_BLOCK) h[c] = bc[c] + src[c];
    __syncthreads();
    const OrdMap m = ord_map(box);
    const long long b0 = (long long)blockIdx.x << ORD_TILE_BITS;
    const long long b1 = min(n, b0 + (1LL << ORD_TILE_BITS));
    for (long long i = b0 + threadIdx.x; i < b1; i += ORD_BLOCK) {
        const unsigned pos = atomicAdd(&h[ord_cell(o, n, i, m)], 1u);
        order[pos] = (int)i;
    }
}

// Exclusive prefix sum of nbins counts in three launches: per-tile sums,
// a scan of the tile sums, per-tile scans with the tile offset.
constexpr int ORD_TILE = 1024;  // counts per scan tile (one block of 1024 threads)

__device__ __forceinline__ unsigned block_exclusive_scan(unsigned v, unsigned* total) {
    __shared__ unsigned warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned x = v;
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0u;
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    const unsigned before = wid > 0 ? warp_sums[wid - 1] : 0u;
    if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
    return before + x - v;
}

__global__ void ord_tile_sums(const unsigned* hist, long long nbins, unsigned* tiles) {
    const long long k = (long long)blockIdx.x * ORD_TILE + threadIdx.x;
    unsigned total;
    block_exclusive_scan(k < nbins ? hist[k] : 0u, &total);
    if (threadIdx.x == 0) tiles[blockIdx.x] = total;
}

__global__ void ord_scan_tiles(unsigned* tiles, int ntiles) {
    // one block: sequential over chunks of 1024 tile sums
    unsigned carry = 0;
    for (int base = 0; base < ntiles; base += ORD_TILE) {
        const int k = base + threadIdx.x;
        const unsigned v = k < ntiles ? tiles[k] : 0u;
        unsigned total;
        const unsigned ex = block_exclusive_scan(v, &total);
        if (k < ntiles) tiles[k] = carry + ex;
        carry += total;
        __syncthreads();
    }
}

__global__ void ord_tile_scan(unsigned* hist, long long nbins, const unsigned* tiles) {
    const long long k = (long long)blockIdx.x * ORD_TILE + threadIdx.x;
    const unsigned ex = block_exclusive_scan(k < nbins ? hist[k] : 0u, nullptr);
    if (k < nbins) hist[k] = tiles[blockIdx.x] + ex;
}

// blocks of the counting passes: whole chunks, so that the count layout is regular
static long long ord_blocks(long long n) {
    const long long chunks = (n + (1LL << ORD_CHUNK_BITS) - 1) >> ORD_CHUNK_BITS;
    return chunks * ORD_TILES_PER_CHUNK;
}

static long long ord_round(long long bytes) { return (bytes + 255) / 256 * 256; }

long long order_scratch_bytes(long long n) {
    const long long nbins = ord_blocks(n) * ORD_CELLS;
    const long long ncells = ord_blocks(n) / ORD_TILES_PER_CHUNK * ORD_CELLS;  // (chunk, cell) totals
    const long long ntiles = (ncells + ORD_TILE - 1) / ORD_TILE;
    return 256 + ord_round(nbins * 4) + ord_round(ncells * 4) + ord_round(n * 4) + ntiles * 4 + 1024;
}

template <typename T>
static cudaError_t build_order_t(const T* o, long long n, void* scratch, int** order_out, int sms, cudaStream_t s) {
    const long long nblk = ord_blocks(n);
    const long long nchunks = nblk / ORD_TILES_PER_CHUNK;
    const long long nbins = nblk * ORD_CELLS, ncells = nchunks * ORD_CELLS;
    const long long ntiles = (ncells + ORD_TILE - 1) / ORD_TILE;
    unsigned char* b = static_cast<unsigned char*>(scratch);
    int* box = reinterpret_cast<int*>(b);
    unsigned* counts = reinterpret_cast<unsigned*>(b + 256);
    unsigned* totals = reinterpret_cast<unsigned*>(b + 256 + ord_round(nbins * 4));
    int* order = reinterpret_cast<int*>(b + 256 + ord_round(nbins * 4) + ord_round(ncells * 4));
    unsigned* tiles =
        reinterpret_cast<unsigned*>(b + 256 + ord_round(nbins * 4) + ord_round(ncells * 4) + ord_round(n * 4));
    const int smem = ORD_CELLS * (int)sizeof(unsigned);
    // the 64 KB shared-memory opt-in, once per device and precision
    static std::atomic<unsigned long long> opted{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 32 ? 1ull << (dev * 2 + (sizeof(T) == 4 ? 0 : 1)) : 0ull;
    if (!bit || !(opted.load(std::memory_order_relaxed) & bit)) {
        e = cudaFuncSetAttribute(ord_count<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(ord_place<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        opted.fetch_or(bit, std::memory_order_relaxed);
    }
    ord_init<<<1, 32, 0, s>>>(box);
    ord_bounds<T><<<sms * 4, 256, 0, s>>>(o, n, box);
    ord_count<T><<<(unsigned)nblk, ORD_BLOCK, smem, s>>>(o, n, box, counts);
    ord_columns<<<(unsigned)((ncells + 255) / 256), 256, 0, s>>>(counts, nchunks, totals);
    ord_tile_sums<<<(unsigned)ntiles, ORD_TILE, 0, s>>>(totals, ncells, tiles);
    ord_scan_tiles<<<1, ORD_TILE, 0, s>>>(tiles, (int)ntiles);
    ord_tile_scan<<<(unsigned)ntiles, ORD_TILE, 0, s>>>(totals, ncells, tiles);
    ord_place<T><<<(unsigned)nblk, ORD_BLOCK, smem, s>>>(o, n, box, counts, totals, order);
    *order_out = order;
    return cudaGetLastError();
}

cudaError_t build_order_f32(const float* o, long long n, void* scratch, int** order, int sms, cudaStream_t s) {
    return build_order_t<float>(o, n, scratch, order, sms, s);
}
cudaError_t build_order_f64(const double* o, long long n, void* scratch, int** order, int sms, cudaStream_t s) {
    return build_order_t<double>(o, n, scratch, order, sms, s);
}

}  // namespace robast
