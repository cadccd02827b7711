// Coherent processing order for the trace: a counting sort of the photon
// indices by (chunk of 4M photons of the input order, cell of the origin in a
// 512 x 512 grid over the origins' x-y bounding box).  Rays of one warp then
// start close together (and, within a chunk of the caller's order, usually
// share a direction), so they walk the same BVH nodes and hit the same
// surfaces and the warp's lanes diverge far less.  The reordered loads and
// stores touch scattered sectors (more DRAM traffic than the I/O itself), but
// on the dish workload the divergence saved outweighs it: measured over grids
// of 16..1024 cells and chunks of 2^16..2^26 photons, this setting gave the
// fastest step.  Results do not depend on the order: every photon keeps its
// index, its random stream and its output slot.
#include <cuda_runtime.h>
#include <stdint.h>

#include "launch.h"

namespace robast {

constexpr int ORD_G = 512;            // grid cells per axis (swept: 16..1024; 512 fastest)
constexpr int ORD_CHUNK_BITS = 22;    // chunks of 4M photons keep the caller's order (swept 16..26)

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

template <typename T>
__device__ __forceinline__ unsigned ord_key(const T* o, long long n, long long i, const int* box) {
    const float x0 = unordered_float(box[0]), x1 = unordered_float(box[1]);
    const float y0 = unordered_float(box[2]), y1 = unordered_float(box[3]);
    const float fx = x1 > x0 ? ((float)o[i] - x0) / (x1 - x0) : 0.0f;
    const float fy = y1 > y0 ? ((float)o[n + i] - y0) / (y1 - y0) : 0.0f;
    int cx = (int)(fx * ORD_G), cy = (int)(fy * ORD_G);
    cx = cx < 0 ? 0 : (cx >= ORD_G ? ORD_G - 1 : cx);
    cy = cy < 0 ? 0 : (cy >= ORD_G ? ORD_G - 1 : cy);
    // serpentine rows keep consecutive cells adjacent
    const int c = cy * ORD_G + ((cy & 1) ? ORD_G - 1 - cx : cx);
    return (unsigned)((i >> ORD_CHUNK_BITS) * (ORD_G * ORD_G) + c);
}

constexpr int ORD_UNROLL = 8;  // photons per thread per iteration: independent atomics in flight

template <typename T>
__global__ void ord_hist(const T* o, long long n, const int* box, unsigned* hist) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; i0 < n; i0 += ORD_UNROLL * stride) {
        unsigned key[ORD_UNROLL];
#pragma unroll
        for (int j = 0; j < ORD_UNROLL; ++j) {
            const long long i = i0 + j * stride;
            key[j] = i < n ? ord_key(o, n, i, box) : 0xffffffffu;
        }
#pragma unroll
        for (int j = 0; j < ORD_UNROLL; ++j)
            if (key[j] != 0xffffffffu) atomicAdd(hist + key[j], 1u);
    }
}

// Exclusive prefix sum of nbins counts in three launches: per-tile sums,
// a scan of the tile sums, per-tile scans with the tile offset.
constexpr int ORD_TILE = 1024;  // bins per tile (one block of 1024 threads)

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

template <typename T>
__global__ void ord_scatter(const T* o, long long n, const int* box, unsigned* offs, int* order) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; i0 < n; i0 += ORD_UNROLL * stride) {
        unsigned pos[ORD_UNROLL];
#pragma unroll
        for (int j = 0; j < ORD_UNROLL; ++j) {
            const long long i = i0 + j * stride;
            pos[j] = i < n ? atomicAdd(offs + ord_key(o, n, i, box), 1u) : 0xffffffffu;
        }
#pragma unroll
        for (int j = 0; j < ORD_UNROLL; ++j)
            if (pos[j] != 0xffffffffu) order[pos[j]] = (int)(i0 + j * stride);
    }
}

long long order_scratch_bytes(long long n) {
    const long long nbins = ((n - 1) >> ORD_CHUNK_BITS) * (long long)(ORD_G * ORD_G) + ORD_G * ORD_G;
    const long long ntiles = (nbins + ORD_TILE - 1) / ORD_TILE;
    return 16 + nbins * 4 + n * 4 + ntiles * 4 + 1024;
}

template <typename T>
static cudaError_t build_order_t(const T* o, long long n, void* scratch, int** order_out, int sms, cudaStream_t s) {
    const long long nbins = ((n - 1) >> ORD_CHUNK_BITS) * (long long)(ORD_G * ORD_G) + ORD_G * ORD_G;
    unsigned char* b = static_cast<unsigned char*>(scratch);
    int* box = reinterpret_cast<int*>(b);
    unsigned* hist = reinterpret_cast<unsigned*>(b + 16);
    int* order = reinterpret_cast<int*>(b + 16 + ((nbins * 4 + 255) / 256) * 256);
    const long long ntiles = (nbins + ORD_TILE - 1) / ORD_TILE;
    unsigned* tiles = reinterpret_cast<unsigned*>(b + 16 + ((nbins * 4 + 255) / 256) * 256 + ((n * 4 + 255) / 256) * 256);
    ord_init<<<1, 32, 0, s>>>(box);
    cudaError_t e = cudaMemsetAsync(hist, 0, nbins * 4, s);
    if (e != cudaSuccess) return e;
    const int grid = sms * 8;
    ord_bounds<T><<<grid, 256, 0, s>>>(o, n, box);
    ord_hist<T><<<grid, 256, 0, s>>>(o, n, box, hist);
    ord_tile_sums<<<(unsigned)ntiles, ORD_TILE, 0, s>>>(hist, nbins, tiles);
    ord_scan_tiles<<<1, ORD_TILE, 0, s>>>(tiles, (int)ntiles);
    ord_tile_scan<<<(unsigned)ntiles, ORD_TILE, 0, s>>>(hist, nbins, tiles);
    ord_scatter<T><<<grid, 256, 0, s>>>(o, n, box, hist, order);
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
