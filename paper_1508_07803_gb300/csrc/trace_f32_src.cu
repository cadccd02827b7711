// float instantiations of the source-mode trace kernel (see trace.cuh): photons generated on the
// device from source groups; the full profile and the concentrator profile (cones and refracting
// faces), and the counting build.
#include <algorithm>

#include "launch.h"

namespace robast {

template <int BLOCK, bool C, bool STAGED, unsigned FEAT>
static cudaError_t launch_one(const TraceArgs<float>& a, int grid, size_t smem, cudaStream_t s) {
    auto k = trace_kernel<float, BLOCK, C, STAGED, true, float, FEAT>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<grid, BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

template <int BLOCK, unsigned FEAT>
static int occupancy_one(size_t smem) {
    auto k = smem ? trace_kernel<float, BLOCK, false, true, true, float, FEAT>
                  : trace_kernel<float, BLOCK, false, false, true, float, FEAT>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, BLOCK, smem) != cudaSuccess) return 0;
    return nb;
}

int trace_blocks_per_sm_f32_src(int block, size_t smem, unsigned prof) {
    const bool cc = prof == FT_CONCENTRATOR;
    switch (block) {
        case 64: return cc ? occupancy_one<64, FT_CONCENTRATOR>(smem) : occupancy_one<64, FT_ALL>(smem);
        case 128: return cc ? occupancy_one<128, FT_CONCENTRATOR>(smem) : occupancy_one<128, FT_ALL>(smem);
        case 256: return cc ? occupancy_one<256, FT_CONCENTRATOR>(smem) : occupancy_one<256, FT_ALL>(smem);
    }
    return 0;
}

template <int BLOCK>
static cudaError_t launch_prof(const TraceArgs<float>& a, int grid, size_t smem, cudaStream_t s, unsigned prof) {
    const bool st = a.stage != 0;
    if (prof == FT_CONCENTRATOR)
        return st ? launch_one<BLOCK, false, true, FT_CONCENTRATOR>(a, grid, smem, s)
                  : launch_one<BLOCK, false, false, FT_CONCENTRATOR>(a, grid, smem, s);
    return st ? launch_one<BLOCK, false, true, FT_ALL>(a, grid, smem, s)
              : launch_one<BLOCK, false, false, FT_ALL>(a, grid, smem, s);
}

cudaError_t launch_trace_f32_src(const TraceArgs<float>& a, int block, int grid, size_t smem, cudaStream_t s,
                                 unsigned prof) {
    const bool st = a.stage != 0;
    if (a.units) {  // counting build (full profile, block 128)
        if (block != 128) return cudaErrorInvalidConfiguration;
        return st ? launch_one<128, true, true, FT_ALL>(a, grid, smem, s)
                  : launch_one<128, true, false, FT_ALL>(a, grid, smem, s);
    }
    switch (block) {
        case 64: return launch_prof<64>(a, grid, smem, s, prof);
        case 128: return launch_prof<128>(a, grid, smem, s, prof);
        case 256: return launch_prof<256>(a, grid, smem, s, prof);
    }
    return cudaErrorInvalidConfiguration;
}

// Origins (x, y) of the photons base .. base + nw - 1 of a source-mode launch, generated exactly
// as the trace kernel generates them and rounded to FP32: the input of the coherent-order sort of
// one chunk (xy: [2 nw], all x then all y; a photon the generator rejects sits at 0, 0).
__global__ void src_origins_kernel(const SrcGroup* groups, int n_groups, long long base, long long nw,
                                   long long first_id, uint2 key, float* xy) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nw;
         i += (long long)gridDim.x * blockDim.x) {
        const long long idx = base + i;
        int lo = 0, hi = n_groups - 1;  // the last group whose first index is <= idx
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (groups[mid].first <= idx)
                lo = mid;
            else
                hi = mid - 1;
        }
        double o[3], lam;
        float x = 0.0f, y = 0.0f;
        if (gen_source(groups[lo], first_id + idx, key, o, &lam)) {
            x = (float)o[0];
            y = (float)o[1];
        }
        xy[i] = x;
        xy[nw + i] = y;
    }
}

cudaError_t launch_src_origins(const SrcGroup* groups, int n_groups, long long base, long long nw,
                               long long first_id, unsigned long long seed, float* xy, int sms, cudaStream_t s) {
    if (nw <= 0) return cudaSuccess;
    const long long need = (nw + 255) / 256;
    const int grid = (int)std::min<long long>(need, (long long)sms * 8);
    src_origins_kernel<<<grid, 256, 0, s>>>(groups, n_groups, base, nw, first_id,
                                            make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)), xy);
    return cudaGetLastError();
}

}  // namespace robast
